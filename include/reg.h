/*
 * reg.h - C ABI of libreg.so: matrix-free NGF + curvature deformable 3D image
 * registration on one GB300 GPU (sm_103a).
 *
 * Model (Budelmann, Koenig, Papenberg, Lellmann, "Fully-deformable 3D image
 * registration in two seconds", BVM 2019):
 *   y* = argmin_y J(y),  J(y) = D_NGF(R, T(P y)) + alpha S_curv(y)   (Sec. 2.1, Eq. 1)
 * D_NGF is the normalized-gradient-field distance of Eq. 2 (Sec. 2.2), S_curv
 * the curvature regulariser (sum of squared Laplacians of the components,
 * Sec. 2.1), P the trilinear grid conversion from the deformation grid to the
 * image grid and P^T its node-centric adjoint (Sec. 2.2, Eq. 3).  J is
 * minimised by L-BFGS inside a coarse-to-fine pyramid (Sec. 2.1).
 *
 * Layout conventions (every array):
 *   - images: m_x * m_y * m_z float32, x fastest: i = x + m_x (y + m_y z);
 *     voxel centre at ((x + 1/2) h_x, (y + 1/2) h_y, (z + 1/2) h_z) mm.
 *   - deformation grid: n_x * n_y * n_z nodes spanning the same box
 *     [0, m_d h_d], node k at k_d H_d, H_d = m_d h_d / (n_d - 1).
 *   - displacement u (and gradients): 3 planes of n_x n_y n_z float32,
 *     component c at [c * n_x n_y n_z + k], in mm; the deformation is
 *     y = node position + u.
 *   - level 0 is the finest (input) resolution; level l is the input
 *     downsampled l times by 2x2x2 means (spacing * 2^l).
 *
 * Errors: every int-returning call returns REG_OK (0) on success, a positive
 * warning, or a negative error code; reg_last_error() then describes it.
 * No call aborts the process.  Device pointers must be valid device memory of
 * the current CUDA device; host pointers plain host memory.
 *
 * Threads and streams: a handle is not thread-safe; all its GPU work is queued
 * on the stream given to reg_create plus one internal side stream (the template
 * pyramid, and the curvature pass that runs beside the NGF pass), forked from
 * and joined back to that stream with events.  Calls that return host values
 * synchronise that stream.  The level graphs (use_graph = 1, and every
 * reg_register_batch) carry their own kernel priorities, whatever the priority
 * of that stream: the curvature pass at the device's lowest stream priority,
 * every other kernel at the highest.
 */
#ifndef REG_H
#define REG_H

#ifdef __cplusplus
extern "C" {
#endif

#define REG_MAX_LEVELS 8
#define REG_MAX_MEM 8
#define REG_MAX_VOXELS 2147483647LL  /* voxels of an image, and 3 x nodes of a deformation grid */
#define REG_MAX_PLANES 65535         /* m_z of an image, n_z of a deformation grid */

#define REG_OK 0
#define REG_WARN_LINESEARCH 1  /* a level ended on a failed Armijo search; u is its last accepted iterate */
#define REG_ERR_ARG (-1)       /* bad argument: NULL, dims < 4, spacing <= 0, node dims < 3, level out of range */
#define REG_ERR_CUDA (-2)      /* a CUDA runtime call failed (message has the CUDA error string) */
#define REG_ERR_OOM (-3)       /* device or pinned host allocation failed */
#define REG_ERR_STATE (-4)     /* call out of order, e.g. evaluation before reg_set_images */
#define REG_ERR_NUMERIC (-5)   /* J or its gradient became NaN/Inf */
#define REG_ERR_TIMEOUT (-6)   /* a bounded device-side wait expired */

typedef struct reg_ctx *reg_handle;

/* Registration parameters.  reg_config_default() fills the values used by the
 * paper's model as read in this library:
 *   tau = rho = 0.01, alpha = 10, c1 = 1e-4, max_backtracks = 20,
 *   tol_grad_rel = 1e-5, tol_j_rel = 1e-7, tol_j_count = 3, levels = 1,
 *   lbfgs_mem = 5, max_iter = 50 on every level, node_dims = 0 (rule m_d/2+1),
 *   start_level = -1 (coarsest), eval_impl = 0 (fused), use_graph = 1, image_dtype = 0,
 *   autotune = 1, fused_tz = 0. */
typedef struct reg_config {
    double tau, rho;      /* NGF edge parameters of Eq. 2 (template, reference), > 0 */
    double alpha;         /* regularisation weight of Eq. 1, >= 0 */
    double c1;            /* Armijo sufficient-decrease constant, in (0, 1) */
    double tol_grad_rel;  /* stop a level when ||grad J|| <= tol_grad_rel * ||grad J(u0)|| */
    double tol_j_rel;     /* ... or when |J_{k-1} - J_k| <= tol_j_rel (1 + |J_0|) */
    int tol_j_count;      /*     for tol_j_count consecutive iterations */
    int levels;           /* pyramid levels, 1 .. REG_MAX_LEVELS */
    int lbfgs_mem;        /* L-BFGS memory m, 1 .. REG_MAX_MEM */
    int max_backtracks;   /* Armijo trials per line search, >= 1 */
    int fixed_iters;      /* 1: only max_iter ends a level (step-for-step comparisons) */
    int start_level;      /* coarsest level solved; -1 = levels - 1 */
    int max_iter[REG_MAX_LEVELS];       /* accepted iterations per level (index = level) */
    int node_dims[REG_MAX_LEVELS][3];   /* deformation grid per level; 0 = m_d / 2 + 1 */
    int eval_impl;        /* 0 fused objective pass; 1 multi-pass (intermediates in HBM,
                             P^T by the gather of Eq. 3); A/B baselines of P^T: 2 multi-pass
                             with an atomic scatter (summation order not fixed), 3 multi-pass
                             with an 8-colour scatter on ratio-2 levels (gather elsewhere) */
    int use_graph;        /* 1: each pyramid level runs as one CUDA graph launch */
    int image_dtype;      /* 0: FP32 images; 1: the fused pass reads BF16 copies of R and T
                             (arithmetic stays FP32; levels without the fused pass use FP32) */
    int autotune;         /* 1: reg_set_images times the z splits of the fused pass that a
                             load model ranks best on each level and keeps the fastest (cached
                             per geometry for the process; the first call of a geometry
                             synchronises the stream); 0: the model's choice */
    int fused_tz;         /* 0: autotune / model; -1: the throughput rule (fewest z steps in
                             total over 2, 4, 8, .. 128) with the fused pass forming the
                             curvature sum per tile, as reg_register_batch computes it;
                             else this z segment length on every level (even, 2 .. 512) */
    int test_expire_wait; /* test hook, 0 in normal use: 1 makes block 0 of the first L-BFGS
                             direction pass of reg_register arm one bulk-copy stage without
                             issuing its copies, so that its bounded wait expires (after about
                             1 s); the level then stops and reg_register returns
                             REG_ERR_TIMEOUT.  Nothing faults: no copy is left in flight. */
    int fused_split[5];   /* all 0: not forced.  Else (l1, n1, l2, n2, lr): on every fused
                             level whose depth is n1 l1 + n2 l2 + lr, z segments of n1 x l1,
                             then n2 x l2, then lr planes (lengths even; before fused_tz) */
    int reserved[1];
} reg_config;

/* Per-registration statistics (filled by reg_register). */
typedef struct reg_stats {
    int levels;
    int iters[REG_MAX_LEVELS];        /* accepted L-BFGS iterations per level */
    int evals[REG_MAX_LEVELS];        /* objective+gradient evaluations per level */
    int level_status[REG_MAX_LEVELS]; /* REG_OK or REG_WARN_LINESEARCH per level */
    double J[REG_MAX_LEVELS];         /* final J per level */
    double J_final, D_final, S_final; /* at the finest level */
    double seconds;                   /* host wall time of the call */
    long long kernel_launches;        /* kernels this call ran on the GPU (graph nodes included) */
    int status;
    double level_seconds[REG_MAX_LEVELS]; /* device time of each level, its prolongation included
                                             (CUDA events on the handle's stream) */
    int tiling[REG_MAX_LEVELS];       /* fused-pass tiling per level: reg_register, the z segment
                                         length (0: multi-pass level); reg_register_batch, the
                                         rule the batch used (0 each pair's own tiling, -1 the
                                         throughput rule, T > 0 one segment length T) */
} reg_stats;

/* Library version (major * 10000 + minor * 100 + patch). */
int reg_version(void);

/* Fill *cfg with the defaults listed above (the model parameters of Sec. 2.1,
 * Eq. 1-2, and the solver's).  cfg must not be NULL. */
void reg_config_default(reg_config *cfg);

/* Create a handle for one registration problem of Sec. 2.1 (Eq. 1) with the
 * parameters of cfg.  cfg is copied (validated here: REG_ERR_ARG on bad values).
 * cuda_stream is a cudaStream_t of the current device, or NULL for the legacy
 * default stream (the stream PyTorch uses unless told otherwise); the caller
 * keeps ownership of a stream it passes.  On success *out owns the handle;
 * free it with reg_destroy.  Allocates no image buffers yet. */
int reg_create(reg_handle *out, const reg_config *cfg, void *cuda_stream);

/* Load a reference R and template T (Sec. 2.1) of dims[3] = (m_x, m_y, m_z)
 * voxels with spacing_mm[3], and build the pyramid of cfg.levels levels on
 * two streams (Sec. 2.2 "Generating the multi-level pyramid").  R and T are
 * device pointers if ptr_is_device, else host pointers; they are copied, the
 * caller keeps ownership.  Each level must keep >= 4 voxels and >= 3 nodes
 * per dimension, an image holds at most REG_MAX_VOXELS voxels and
 * REG_MAX_PLANES planes, and a deformation grid at most REG_MAX_VOXELS / 3
 * nodes and REG_MAX_PLANES node planes (the kernels index with 32-bit
 * integers and launch one grid row per plane); REG_ERR_ARG otherwise, and the
 * handle keeps its previous images.  Replaces previous images. */
int reg_set_images(reg_handle h, const float *R, const float *T, const int dims[3],
                   const double spacing_mm[3], int ptr_is_device);

/* Geometry of one pyramid level (Sec. 2.2 "Generating the multi-level
 * pyramid"; the deformation grid of Sec. 2.2 "Grid conversion"): image dims,
 * node dims, voxel spacing and node spacing (mm).  Any output pointer may be
 * NULL. */
int reg_level_info(reg_handle h, int level, int img_dims[3], int node_dims[3],
                   double spacing_mm[3], double node_spacing_mm[3]);

/* Tiling of the fused objective pass on a level (no counterpart in the paper,
 * which uses separate kernels): *tz = the longest z segment (output planes per
 * CTA, chosen by the autotuner, cfg.fused_split, cfg.fused_tz or the load
 * model), *tiles = CTAs per evaluation.  Both 0 on levels the multi-pass
 * kernels serve.  Any output pointer may be NULL. */
int reg_level_tiling(reg_handle h, int level, int *tz, int *tiles);

/* (No counterpart in the paper.)  The load model's z split of the fused pass
 * for an image of dims[3] voxels (each even) on a GPU with num_sms SMs,
 * without a GPU or a handle: the split a handle uses when cfg.autotune = 0
 * (the autotuner times it among others).
 * split[5] as in cfg.fused_split; *model_steps (nullable) = the model's
 * duration in pipeline steps of one CTA.  REG_ERR_ARG for odd or < 4 dims or
 * num_sms < 1. */
int reg_fused_split_plan(const int dims[3], int num_sms, int split[5], double *model_steps);

/* (No counterpart in the paper.)  Tile geometry of the fused pass, host only:
 * *ox, *oy = output voxel columns of a tile along x and y (a tile computes a
 * 2-voxel halo around them), *ctas_per_sm = the pass's CTAs resident per SM
 * (the load model's slots per SM).  Any pointer may be NULL.  Returns REG_OK. */
int reg_fused_tile_shape(int *ox, int *oy, int *ctas_per_sm);

/* The per-dimension grid-conversion tables that reg_set_images uploads for one
 * axis of m voxels of spacing h and n nodes (host only, no GPU; Sec. 2.2,
 * Eq. 3: the index sets and weights of P and P^T are fixed beforehand and
 * separately for each dimension).  With voxel centres at t_i = (i + 1/2) h / H
 * in node units, H = m h / (n - 1), and the hat function phi(t) = max(0, 1 - |t|):
 *   P:   k0[i] = floor(t_i) clamped to 0 .. n - 2 and w1[i] = t_i - k0[i]
 *        (voxel i takes 1 - w1 of node k0 and w1 of node k0 + 1); m entries each;
 *   P^T: node k gathers cnt[k] voxels from first[k] on, voxel first[k] + j with
 *        weight w[k * max_w + j] = phi(t_{first[k] + j} - k) > 0 (zero-padded to
 *        max_w); n entries in first and cnt, n * max_w in w.
 * Caller-owned host arrays; any may be NULL to skip it.  *needed_w (nullable)
 * receives the largest cnt.  REG_ERR_ARG for m < 4, n < 3, h not finite and
 * > 0, or max_w below the largest cnt when w is given. */
int reg_axis_tables(int m, double h, int n, int *k0, float *w1, int *first, int *cnt, float *w, int max_w,
                    int *needed_w);

/* (No counterpart in the paper.)  The z split of the fused pass on a level,
 * in the form of cfg.fused_split: split[5] = (l1, n1, l2, n2, lr), n1
 * segments of l1 planes, then n2 of l2, then lr planes (0: no remainder),
 * every tile column alike.  All 0 on levels the multi-pass kernels serve.
 * REG_ERR_STATE before reg_set_images. */
int reg_level_split(reg_handle h, int level, int split[5]);

/* Copy pyramid image `which` (0 = R, 1 = T) of a level (Sec. 2.2 "Generating
 * the multi-level pyramid": 2 x 2 x 2 means) into out
 * (m_x m_y m_z floats; device pointer if out_is_device). */
int reg_get_level_image(reg_handle h, int level, int which, float *out, int out_is_device);

/* One evaluation of J (Eq. 1) and grad_u J at a level, matrix-free
 * (Sec. 2.2 "Evaluating the objective function": P, NGF and its chain-rule
 * gradient, P^T by the gather of Eq. 3, plus alpha times the curvature term).
 * u_dev, grad_dev: device pointers, 3 planes of the level's node count
 * (borrowed; grad_dev is overwritten).  J, D, S: host pointers (any may be
 * NULL) receiving J, D_NGF and S_curv in double; the call synchronises the
 * handle's stream when any of them is non-NULL. */
int reg_eval_objective_grad(reg_handle h, int level, const float *u_dev, float *grad_dev,
                            double *J, double *D, double *S);

/* Device time (ms) of the NGF pass of the last reg_eval_objective_grad call on
 * this handle: the fused kernel (or the multi-pass NGF kernels), timed with
 * CUDA events on the handle's stream around its launch; the curvature and
 * gradient-assembly kernels are not included.  Synchronises on that event.
 * REG_ERR_STATE before the first evaluation.  A profiling aid (the paper
 * reports whole-registration times only, Sec. 3). */
int reg_last_ngf_ms(reg_handle h, double *ms);

/* Allocation-free evaluation: the same J, D_NGF, S and grad_u J as
 * reg_eval_objective_grad computes at one resolution, for callers that must not
 * allocate device memory while they run - code hosted by a framework that owns
 * all device memory through its own pool and budget, or a latency-bound loop
 * that cannot go through cudaMalloc / cudaFree (which may synchronise the
 * device).  It has no counterpart in the paper: it is an interface of this library.
 *   R, T: device images, dims[3] = (m_x, m_y, m_z), each even and >= 4 (the
 *     deformation grid is m_d / 2 + 1 nodes per dimension), spacing_mm[3] > 0;
 *     R must be 8-byte aligned (it is read two voxels at a time; any cudaMalloc
 *     pointer is), else REG_ERR_ARG;
 *   u, grad: device, 3 planes of the node count (grad is overwritten);
 *   tau, rho > 0, alpha >= 0: the same parameters as reg_config's tau, rho and
 *     alpha for reg_eval_objective_grad;
 *   jds: device, 3 doubles receiving J, D and S;
 *   cuda_stream: a cudaStream_t, or NULL for the legacy default stream.
 * Every buffer is the caller's.  The working memory is one fixed 20.5 MiB array
 * in the library's device image, held by every GPU that loads the library until
 * the process exits; it fits images up to about 136^3 voxels (a 128^3 pair
 * needs at most 12.3 MiB), and larger sizes are rejected with REG_ERR_ARG before
 * anything is launched, as is any side above 4096 voxels.  No call allocates
 * memory.  The first call on each device looks up the array's device address
 * and sets a kernel attribute for that device (again on the first call after
 * the device's context was reset, e.g. by cudaDeviceReset): make that first
 * call before any stream capture.  All calls share
 * the array and every call overwrites what it reads, so calls that may overlap
 * on the GPU (different streams or threads) race and must be serialised by the
 * caller.  Returns REG_OK, REG_ERR_ARG or REG_ERR_CUDA; reg_last_error(NULL)
 * describes a failure.  Nothing is synchronised. */
int reg_eval_objective_grad_noalloc(const float *R, const float *T, const int dims[3],
                                    const double spacing_mm[3], const float *u, float *grad,
                                    double tau, double rho, double alpha, double *jds,
                                    void *cuda_stream);

/* Nodal trilinear prolongation (Sec. 2.1 multilevel) of a displacement from
 * level `level_coarse` to level_coarse - 1.  Device pointers, 3 planes each. */
int reg_prolong(reg_handle h, int level_coarse, const float *uc_dev, float *uf_dev);

/* p = -H g for the L-BFGS matrix H built from `count` pairs (Sec. 2.1, L-BFGS of
 * Nocedal 1980) with H0 = gamma I, gamma = s'y / y'y of the newest pair, using
 * the same device kernels as reg_register.  S_dev, Y_dev: count * n floats,
 * pair j at offset j * n, oldest first; g_dev, p_dev: n floats.  All device
 * pointers; p_dev is overwritten.  count in 0 .. lbfgs_mem; with count = 0
 * p = -g min_d H_d / ||g||_inf for the finest level's node spacing H. */
int reg_lbfgs_direction(reg_handle h, long long n, int count, const float *S_dev,
                        const float *Y_dev, const float *g_dev, float *p_dev);

/* Full multilevel registration (Sec. 2.1-2.2): L-BFGS with Armijo
 * backtracking at every level from start_level to 0, prolongating between
 * levels.  u_init: displacement on the start level's node grid (same memory
 * kind as u_out), or NULL for zero.  u_out: the finest level's displacement,
 * device pointer if out_is_device else host.  st (nullable) receives the
 * statistics.  Returns REG_OK, REG_WARN_LINESEARCH, or an error. */
int reg_register(reg_handle h, float *u_out, int out_is_device, const float *u_init, reg_stats *st);

/* Register n pairs together (many pairs of uneven size, Sec. 2.1-2.2 per
 * pair): each hs[i] is a handle with its images set; all share the number of
 * levels, the start level, image_dtype and the device, and every level must be a
 * ratio-2 grid served by the fused pass (even dims, default node counts,
 * eval_impl 0).  Per pyramid level the pairs iterate in lock step inside one
 * CUDA graph launch: each kernel of an iteration runs once for the whole batch
 * over a work list of (pair, tile / block) items, and pairs that have finished
 * their level or their line search skip their items.  Every pair runs exactly
 * the computation of reg_register with its own configuration, so its result is
 * the one reg_register gives when the pair's handle tiles the fused pass the
 * same way: the batch keeps every SM busy, so it tiles each level by the
 * throughput rule and forms the curvature sum inside the fused pass
 * (cfg.fused_tz = -1) whatever the handle's own registrations use.  u_out[i]: the finest displacement of pair i
 * (device pointers if out_is_device, else host); stats (nullable) receives n
 * entries (kernel_launches counts the launches of the whole batch).  Work runs
 * on hs[0]'s stream, as one CUDA graph per level, or queued from the host when
 * hs[0]'s cfg.use_graph is 0; the call synchronises the stream.  Returns REG_OK,
 * REG_WARN_LINESEARCH (some pair), or an error (argument errors are described
 * by reg_last_error(NULL), CUDA errors by reg_last_error(hs[0])). */
int reg_register_batch(reg_handle *hs, int n, float **u_out, int out_is_device, reg_stats *stats);

/* Release all device memory, streams and graphs of the handle.  NULL-safe.
 * Returns REG_OK. */
int reg_destroy(reg_handle h);

/* Message of the last failed call on this handle (or of the last failed
 * reg_create on this thread when h is NULL).  Never NULL; valid until the
 * next call on the handle. */
const char *reg_last_error(reg_handle h);

#ifdef __cplusplus
}
#endif

#endif /* REG_H */
