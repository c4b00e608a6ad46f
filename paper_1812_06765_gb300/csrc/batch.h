// Batched registration: one descriptor per pair and pyramid level, read by
// the batched kernels, which walk prefix-sum work lists over all pairs.
#pragma once

#include "internal.h"

// Arguments of the fused objective pass over one pair (k_ngf_fused.cu).
struct FusedArgs {
    LevelGeom g;
    const void *T, *R;      // images, elements of the kernel's IMG type (float or bf16)
    const float4 *Rn;       // R's normalized gradient field (FP32 images of a handle; else null)
    const float *ub, *dir;
    const double *t_dev;
    float tau, rho;
    FusedSplit split;       // z segments (the same for every tile column)
    int ntx, nty;           // tile columns
    float *part;            // per segment (z order): [tile column][len/2 + 1][NE]
    double *partials;       // D block partials, one per tile
    float *w;               // curvature Laplacian of every node (3 planes), written by the owning tiles
    double *partials_S;     // sums of w^2 over each tile's nodes, one per tile
};

struct PairLevel {
    // objective evaluation
    FusedArgs fa_init;      // at u (level start)
    FusedArgs fa_trial;     // at u + t pdir, t read from the pair's state
    LevelGeom geom;
    float *w;               // curvature Laplacian scratch
    double *pS;             // curvature block partials (after the fused-pass partials)
    int nD, nS;             // block partials of D and of S (= curvature blocks)
    int ngather;            // gather blocks (GATHER_NODES nodes of one plane each)
    double hbar_half, alpha, hy_half;
    float alpha_hy;
    double *scal, *scal_t;  // [J, D, S] at u and at the trial point
    // L-BFGS
    LbfgsState *st;
    long long n, stride;    // vector length, ring slot stride
    float *u, *g, *gt, *pdir, *P, *Y;
    float *lpart;           // vector-pass block partials (FP32)
    float2 *lgpart;         // their group sums (double-float)
    unsigned *lcnt;         // arrival counters of the groups
    int nchunks;            // blocks of the vector passes
    int ntx, nty;           // fused tile columns (also inside fa_*)
    int gbx;                // gather blocks per node plane
};

// prefix sums of per-pair item counts: item i belongs to pair p with
// off[p] <= i < off[p + 1]
struct WorkLists {
    int *tiles;             // fused-pass tiles
    int *nodes;             // gather blocks
    int *chunks;            // vector-pass blocks
    int *curv;              // curvature blocks
    int total_tiles, total_nodes, total_chunks, total_curv;
};

__device__ __forceinline__ int find_pair(const int *__restrict__ off, int npairs, int item)
{
    int lo = 0, hi = npairs;   // off[lo] <= item < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= item)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// batched launchers (mode 0: objective at u, 1: at the trial point of pairs still searching)
cudaError_t launch_fused_batch(const PairLevel *pl, const int *tile_off, int npairs, int total, int mode, bool bf16,
                               int grid, int device, cudaStream_t s);
cudaError_t launch_gather_batch(const PairLevel *pl, const int *off, int npairs, int total, int mode, int grid,
                                cudaStream_t s);
cudaError_t launch_finalize_batch(const PairLevel *pl, int npairs, int mode, cudaStream_t s);
// step 0: norms of g, 1: direction, 2: its p0 redo, 3: accept
cudaError_t launch_lb_vector_batch(const PairLevel *pl, const int *chunk_off, int npairs, int total, int step,
                                   int grid, cudaStream_t s);
cudaError_t launch_lb_control_batch(const PairLevel *pl, int npairs, int phase, cudaStream_t s);
// sets handle h to "any pair iterates" (which 0) or "any pair searches" (which 1);
// counts its runs in counters[which]
cudaError_t launch_batch_condition(const PairLevel *pl, int npairs, int which, unsigned long long h, int *counters,
                                   cudaStream_t s);
void fused_tiling(const Level &L, int num_sms, FusedSplit *split, int *ntx, int *nty);
// arguments of the fused pass of one handle's level; *ntiles = its tiles
FusedArgs fused_args(const reg_ctx *c, int level, const float *ub, const float *dir, const double *t_dev,
                     double *partials, int *ntiles);
