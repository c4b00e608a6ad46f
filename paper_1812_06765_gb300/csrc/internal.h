// Host-side internals of libreg.so: the handle, per-level buffers, launchers.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <string>

#include "../../include/reg.h"
#include "common.cuh"
#include "lbfgs_state.h"

// z segmentation of the fused pass, the same for every tile column: from
// plane 0, n1 segments of l1 planes, then n2 of l2, then one of lr (lr = 0:
// none).  Lengths are even and add up to the level's depth, so segments of
// different lengths can balance the SMs' load where equal ones leave a
// partial last wave.
struct FusedSplit {
    int l1 = 0, n1 = 0, l2 = 0, n2 = 0, lr = 0;
    __host__ __device__ int count() const { return n1 + n2 + (lr > 0 ? 1 : 0); }
    __host__ __device__ bool valid() const { return count() > 0; }
    // segment s in z order: first plane and length
    __host__ __device__ void seg(int s, int &z0, int &len) const
    {
        if (s < n1) {
            z0 = s * l1;
            len = l1;
        } else if (s < n1 + n2) {
            z0 = n1 * l1 + (s - n1) * l2;
            len = l2;
        } else {
            z0 = n1 * l1 + n2 * l2;
            len = lr;
        }
    }
    // node planes of one tile (length / 2 + 1) summed over the segments before s
    __host__ __device__ long long planes_before(int s) const
    {
        long long p = (long long)(s < n1 ? s : n1) * (l1 / 2 + 1);
        if (s > n1)
            p += (long long)(s - n1 < n2 ? s - n1 : n2) * (l2 / 2 + 1);
        if (s > n1 + n2 && lr > 0)
            p += lr / 2 + 1;
        return p;
    }
    __host__ __device__ int longest() const
    {
        int m = n1 > 0 ? l1 : 0;
        if (n2 > 0 && l2 > m)
            m = l2;
        return lr > m ? lr : m;
    }
    bool operator==(const FusedSplit &o) const
    {
        return l1 == o.l1 && n1 == o.n1 && l2 == o.l2 && n2 == o.n2 && lr == o.lr;
    }
};

// Image, table and geometry buffers of one pyramid level.
struct Level {
    int m[3];
    int n[3];
    double h[3];
    double H[3];
    long long nv, nn;
    float *R = nullptr, *T = nullptr;        // device images
    // read by the fused pass: T with a 2-voxel zero border on every side (dims m + 4), FP32
    // (image_dtype 0) or BF16 (Tb, image_dtype 1, beside the BF16 copy Rb of R)
    float *Tp = nullptr;
    __nv_bfloat16 *Rb = nullptr, *Tb = nullptr;
    // read by the fused pass beside Tp: R's normalized gradient field (b / ||b||_rho,
    // rho / ||b||_rho) per voxel, b the central-difference gradient; zero off the interior
    float4 *Rn = nullptr;
    int *pk0[3] = {nullptr, nullptr, nullptr};
    float *pw1[3] = {nullptr, nullptr, nullptr};
    int *tfirst[3] = {nullptr, nullptr, nullptr};
    int *tcnt[3] = {nullptr, nullptr, nullptr};
    float *tw[3] = {nullptr, nullptr, nullptr};
    int tmaxw[3] = {0, 0, 0};
    // prolongation from level + 1 onto this level's nodes
    int *qk0[3] = {nullptr, nullptr, nullptr};
    float *qw1[3] = {nullptr, nullptr, nullptr};
    FusedSplit split;   // z segments of the fused pass (not valid: not chosen yet)
    LevelGeom geom() const;
};

// Scratch of one objective evaluation, sized for the finest level.
struct EvalScratch {
    float *Tw = nullptr;    // deformed template (multi-pass)
    float *dT = nullptr;    // 3 planes: interpolant gradient (multi-pass)
    float *v = nullptr;     // 3 planes: d psi / d grad Tw (multi-pass)
    float *r = nullptr;     // 3 planes: g * grad T (multi-pass)
    float *w = nullptr;     // 3 node planes: masked Laplacian of u
    float *part = nullptr;  // fused pass: per-tile partial node sums
    double *partials = nullptr;   // block partial sums
    int max_partials = 0;
    double *scal = nullptr;       // [J, D, S] on the device
    size_t part_floats = 0;
};

// Buffers of the device L-BFGS, sized for the finest level.
struct LbfgsBuffers {
    long long n = 0;
    int slots = 0;
    float *u = nullptr, *pdir = nullptr, *g = nullptr, *gt = nullptr;
    float *P = nullptr, *Y = nullptr;   // slots * n each
    float *partials = nullptr;          // FP32 block partials of the vector passes
    int max_partials = 0;
    float2 *gpart = nullptr;            // their group sums, double-float (hi, lo)
    unsigned *cnt = nullptr;            // their arrival counters
    int cnt_len = 0;
    unsigned *gbar = nullptr;           // [arrivals, generation, flags] of the whole-level kernel's grid barrier
    LbfgsState *st = nullptr;           // device
    LbfgsState *st_host = nullptr;      // pinned mirror
    double *scal_t = nullptr;           // [J, D, S] of the trial point
};

struct reg_ctx {
    reg_config cfg;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream for graph capture
    bool own_stream = false;
    cudaEvent_t ev_side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;   // curvature pass beside the NGF pass
    cudaEvent_t kev[2] = {nullptr, nullptr};   // around the NGF pass of reg_eval_objective_grad
    bool time_ngf = false;                     // record kev in the next launch_eval (never while capturing)
    bool kev_valid = false;
    int device = 0;
    int num_sms = 0;
    int levels = 0;
    bool have_images = false;
    long long launches = 0;   // kernels queued by this handle (for reg_stats)
    Level L[REG_MAX_LEVELS];
    EvalScratch es;
    LbfgsBuffers lb;
    std::string err;
    // CUDA graph of one L-BFGS iteration per level (built lazily)
    cudaGraphExec_t iter_graph[REG_MAX_LEVELS] = {};
    cudaGraphExec_t init_graph[REG_MAX_LEVELS] = {};
    // events at the level boundaries of reg_register (created on first use)
    cudaEvent_t lev_ev[REG_MAX_LEVELS + 1] = {};
};

// status helpers
int set_err(reg_ctx *c, int code, const char *fmt, ...);
int cuda_err(reg_ctx *c, cudaError_t e, const char *what);

#define CK(call)                                                          \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return cuda_err(c, _e, #call);             \
    } while (0)

// The curvature Laplacian pass: blocks of 32 x 8 nodes over CURV_ZB node
// planes, one FP64 partial of S per block.
#define CURV_ZB 1
inline int curv_zchunks(int nz) { return (nz + CURV_ZB - 1) / CURV_ZB; }

// launchers (return cudaError_t of the launch)
cudaError_t launch_restrict(const float *src, const int m[3], float *dst, cudaStream_t s);
cudaError_t launch_to_bf16(const float *src, __nv_bfloat16 *dst, long long n, cudaStream_t s);
// the zero-bordered copy of a volume of dims m read by the fused pass (dims m + 4)
long long padded_voxels(const int m[3]);
cudaError_t launch_pad_template(const float *src, const int m[3], float *dst, cudaStream_t s);
cudaError_t launch_pad_template(const float *src, const int m[3], __nv_bfloat16 *dst, cudaStream_t s);
cudaError_t launch_ref_normal_field(const Level &L, double rho, cudaStream_t s);
cudaError_t launch_prolong(const Level &coarse, const Level &fine, const float *uc, float *uf, cudaStream_t s);

// objective + gradient at u_base + t_scale * dir (dir may be NULL: plain u_base);
// t_scale is read on the device from *t_dev when dir != NULL.
// Writes grad (3 node planes) and scal_out[0..2] = J, D, S (device).
// ctl_phase >= 0: the final reduction also runs that L-BFGS control phase.
cudaError_t launch_eval(reg_ctx *c, int level, const float *u_base, const float *dir, const double *t_dev,
                        float *grad, double *scal_out, int ctl_phase, cudaStream_t s);
cudaError_t launch_gather_fin(reg_ctx *c, int level, const float *w, float alpha_hy, float *grad, int nD,
                              const double *pS, int nS, double *scal, int phase, cudaStream_t s);
cudaError_t launch_finalize_ctl(reg_ctx *c, const double *pD, int nD, const double *pS, int nS, double hbar_half,
                                double alpha, double hy_half, double *scal, int phase, cudaStream_t s);

// L-BFGS device steps (k_lbfgs.cu)
cudaError_t lbfgs_launch_init(reg_ctx *c, int level, cudaStream_t s);
cudaError_t lbfgs_launch_direction_level(reg_ctx *c, int level, cudaStream_t s);
cudaError_t lbfgs_launch_trial(reg_ctx *c, int level, cudaStream_t s);
cudaError_t lbfgs_launch_accept_level(reg_ctx *c, int level, cudaStream_t s);
// the whole loop of a small level as one cooperative kernel (after lbfgs_launch_init)
bool lbfgs_level_loop_ok(reg_ctx *c, int level);
cudaError_t lbfgs_launch_level_loop(reg_ctx *c, int level, cudaStream_t s);
void lbfgs_set_graph_handles(unsigned long long h_ls, unsigned long long h_iter, unsigned long long h_redo);
unsigned long long lbfgs_graph_handle_ls();
cudaError_t lbfgs_launch_direction(reg_ctx *c, int level, cudaStream_t s);
cudaError_t lbfgs_launch_redo(reg_ctx *c, int level, cudaStream_t s);
void lbfgs_state_reset_host(LbfgsState *st, const reg_config &cfg, int max_iter, double Hmin);
cudaError_t lbfgs_direction_standalone(reg_ctx *c, long long n, int count, const float *S, const float *Y,
                                       const float *g, float *p, double Hmin, cudaStream_t s);
int eval_partials_needed(const Level &L);
int num_blocks_for(reg_ctx *c, long long n, int threads);
// raises the shared-memory limit of the streamed L-BFGS vector passes on a device (once)
cudaError_t lbfgs_kernels_setup(int device);

// objective pass variants (k_ngf_fused.cu, k_ngf_multipass.cu)
bool fused_eligible(const Level &L);
size_t fused_part_floats(const Level &L, int num_sms);
bool fused_tz_valid(int tz);
// output columns of a fused tile along x and y, and the pass's resident CTAs per SM
void fused_tile_shape(int *ox, int *oy, int *ctas_per_sm);
inline int fused_slots(int num_sms)   // CTAs of the fused pass resident on the whole GPU
{
    int ox, oy, k;
    fused_tile_shape(&ox, &oy, &k);
    return k * num_sms;
}
int fused_tz_throughput(const Level &L);
// tz-plane segments and the remainder
FusedSplit fused_split_uniform(int tz, int mz);
// L.split, or the load model's choice if none has been set
FusedSplit fused_split(const Level &L, int num_sms);
// the load model's choice for an image of m voxels (host only)
FusedSplit fused_split_plan(const int m[3], int num_sms, double *model_steps);
// z segment length and tile grid the fused pass uses on the level
void fused_tiling(const Level &L, int num_sms, FusedSplit *split, int *ntx, int *nty);
// times the z splits the load model ranks best on the level's images at
// u_zero (3 node planes of zeros) and keeps the fastest in L.split; cached per
// geometry
cudaError_t fused_autotune(reg_ctx *c, int level, const float *u_zero, cudaStream_t s);
cudaError_t launch_ngf_fused(reg_ctx *c, int level, const float *ub, const float *dir, const double *t_dev,
                             float *grad, double *partials, int *n_partials, cudaStream_t s);
cudaError_t launch_ngf_multipass(reg_ctx *c, int level, const float *ub, const float *dir, const double *t_dev,
                                 float *grad, double *partials, int *n_partials, cudaStream_t s);

cudaError_t launch_gather_grad(reg_ctx *c, int level, const float *w, float alpha_hy, float *grad, cudaStream_t s);
// gather grids from this many blocks up run the final reduction beside the gather (side stream)
constexpr long long GATHER_SPLIT_BLOCKS = 4096;
// The node gather of the fused pass: a block takes GATHER_NODES consecutive
// nodes of one node plane (runs along x, then y); grid = runs per plane x planes.
constexpr int GATHER_NODES = 256;
inline int gather_runs_per_plane(const int n[3]) { return (n[0] * n[1] + GATHER_NODES - 1) / GATHER_NODES; }
inline dim3 gather_grid(const int n[3]) { return dim3(gather_runs_per_plane(n), n[2], 1); }
inline long long gather_blocks(const int n[3]) { return (long long)gather_runs_per_plane(n) * n[2]; }

cudaError_t build_level_graph(reg_ctx *c, int level, cudaGraphExec_t *out);
// the curvature Laplacian kernels that run beside the NGF pass (to tell their graph nodes apart)
const void *curv_w_kernel();
// kernel nodes of g: low_func at the lowest priority, the others at the highest
cudaError_t set_graph_kernel_priorities(cudaGraph_t g, const void *low_func);
int eval_kernel_count(const reg_ctx *c, int level);

// the fused pass serves levels whose grids have ratio exactly 2; others use the multi-pass kernels
inline bool use_fused(const reg_ctx *c, int level)
{
    return c->cfg.eval_impl == 0 && fused_eligible(c->L[level]);
}

// Levels of at most WHOLE_LEVEL_MAX_NODES nodes are small: a level graph runs
// them as one cooperative kernel (every iteration of the level, a grid barrier
// between phases) where the fused pass serves them, their images are FP32 and
// the device supports cooperative launches (lbfgs_launch_level_loop).  Larger
// levels lose more to the kernel's single 200 KB block per SM (one fused-pass
// CTA per SM instead of two) than they gain (a 65^3-node level took 1.3x).
constexpr long long WHOLE_LEVEL_MAX_NODES = 40000;
inline bool small_level(const reg_ctx *c, int level) { return c->L[level].nn <= WHOLE_LEVEL_MAX_NODES; }

// Whether the fused pass forms the curvature Laplacian itself (one S partial
// per tile) instead of a curvature kernel beside it: the batched form always
// does (its persistent grid leaves no SM for a pass beside it), a single
// registration does with the batch's tiling rule (cfg.fused_tz = -1), so that
// it computes exactly what the batch computes for that pair, and on small
// levels, whose whole-level kernel has no second stream (queued from the host
// they take the same arithmetic).
inline bool fused_curv_in_pass(const reg_ctx *c, int level)
{
    return c->cfg.fused_tz == -1 || small_level(c, level);
}

// P^T of the multi-pass path: 0 node-centric gather (Eq. 3; eval_impl 0 and 1),
// 1 atomic scatter (eval_impl 2), 2 8-colour scatter (eval_impl 3 on ratio-2
// levels; other levels use the gather)
inline int mp_pt_variant(const reg_ctx *c, int level)
{
    if (c->cfg.eval_impl == 2)
        return 1;
    if (c->cfg.eval_impl == 3 && fused_eligible(c->L[level]))
        return 2;
    return 0;
}
