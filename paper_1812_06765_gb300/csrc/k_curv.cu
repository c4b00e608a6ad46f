// Curvature regulariser (Sec. 2.1: penalises (Laplace y_c)^2, Fischer and
// Modersitzki) and the final assembly J = D + alpha S (Eq. 1).
//
//   w_c = mask_interior * L u_c          (7-point Laplacian, node spacing H)
//   S   = hbar_y / 2 sum_c sum_k w_c^2
//   grad_c J += alpha hbar_y L^T w_c     (the symmetric stencil gathered over
//                                         the zero-extended w)
// Both passes are node-parallel, one thread per node and all 3 components.
#include "batch.h"
#include "internal.h"
#include "ngf_math.cuh"

namespace {

// block (bx, by, bzc) of 32 x 8 nodes over the CURV_ZB node planes from
// bzc * CURV_ZB; its S partial goes to partials[lin]
__device__ __forceinline__ void curv_w_body(const LevelGeom &g, const float *__restrict__ ub,
                                            const float *__restrict__ dir, const double *__restrict__ t_dev,
                                            float *__restrict__ w, double *__restrict__ partials, int bx, int by,
                                            int bzc, int lin)
{
    __shared__ double sm[8];
    const int x = bx * blockDim.x + threadIdx.x;
    const int y = by * blockDim.y + threadIdx.y;
    const bool in = x < g.n[0] && y < g.n[1];
    const float t = dir ? (float)__ldg(t_dev) : 0.f;
    const size_t st[3] = {1, (size_t)g.n[0], (size_t)g.n[0] * g.n[1]};
    const bool inxy = x >= 1 && y >= 1 && x <= g.n[0] - 2 && y <= g.n[1] - 2;
    const int z1 = min(g.n[2], (bzc + 1) * CURV_ZB);
    float acc = 0.f;
    if (in)
        for (int z = bzc * CURV_ZB; z < z1; z++) {
            const size_t k = x + (size_t)g.n[0] * (y + (size_t)g.n[1] * z);
            const bool interior = inxy && z >= 1 && z <= g.n[2] - 2;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                float lap = 0.f;
                if (interior) {
                    const float *u = ub + c * g.nn;
                    const float *d = dir ? dir + c * g.nn : nullptr;
                    float u0 = node_value(u, d, t, k);
#pragma unroll
                    for (int e = 0; e < 3; e++)
                        lap = fmaf(node_value(u, d, t, k + st[e]) - 2.f * u0 + node_value(u, d, t, k - st[e]),
                                   g.iH2[e], lap);
                }
                w[c * g.nn + k] = lap;
                acc = fmaf(lap, lap, acc);
            }
        }
    double s = block_sum_to_f64(acc, sm);
    if (linear_tid() == 0)
        partials[lin] = s;
}

__global__ void __launch_bounds__(256) k_curv_w(LevelGeom g, const float *__restrict__ ub,
                                                const float *__restrict__ dir, const double *__restrict__ t_dev,
                                                float *__restrict__ w, double *__restrict__ partials)
{
    curv_w_body(g, ub, dir, t_dev, w, partials, blockIdx.x, blockIdx.y, blockIdx.z, linear_bid());
}

__global__ void __launch_bounds__(256) k_curv_grad(LevelGeom g, const float *__restrict__ w, float alpha_hy,
                                                   float *__restrict__ grad)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int z = blockIdx.z;
    if (x >= g.n[0] || y >= g.n[1])
        return;
    size_t k = x + (size_t)g.n[0] * (y + (size_t)g.n[1] * z);
    size_t st[3] = {1, (size_t)g.n[0], (size_t)g.n[0] * g.n[1]};
    int j[3] = {x, y, z};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float *wc = w + c * g.nn;
        float w0 = __ldg(wc + k);
        float s = 0.f;
#pragma unroll
        for (int e = 0; e < 3; e++) {
            float lo = j[e] > 0 ? __ldg(wc + k - st[e]) : 0.f;
            float hi = j[e] < g.n[e] - 1 ? __ldg(wc + k + st[e]) : 0.f;
            s = fmaf(lo + hi - 2.f * w0, g.iH2[e], s);
        }
        grad[c * g.nn + k] = fmaf(alpha_hy, s, grad[c * g.nn + k]);
    }
}

__global__ void __launch_bounds__(512) k_finalize(const double *__restrict__ pD, int nD,
                                                  const double *__restrict__ pS, int nS, double hbar_half,
                                                  double alpha, double hy_half, double *__restrict__ scal)
{
    finalize_body(pD, nD, pS, nS, hbar_half, alpha, hy_half, scal);
}

// Batched forms over all pairs of a level.  Mode 0: at u; mode 1: at the trial
// point, only for pairs still searching.
__device__ __forceinline__ bool batch_skip(const PairLevel &P, int mode)
{
    return mode == 1 && !(P.st->active && P.st->ls_continue);
}


__global__ void __launch_bounds__(512) k_finalize_batch(const PairLevel *__restrict__ pl, int mode)
{
    const PairLevel &P = pl[blockIdx.x];
    if (batch_skip(P, mode))
        return;
    finalize_body(P.fa_init.partials, P.nD, P.pS, P.nS, P.hbar_half, P.alpha, P.hy_half, mode ? P.scal_t : P.scal);
}

}  // namespace

const void *curv_w_kernel() { return reinterpret_cast<const void *>(k_curv_w); }


cudaError_t launch_finalize_batch(const PairLevel *pl, int npairs, int mode, cudaStream_t s)
{
    k_finalize_batch<<<npairs, 512, 0, s>>>(pl, mode);
    return cudaGetLastError();
}

cudaError_t launch_eval(reg_ctx *c, int level, const float *ub, const float *dir, const double *t_dev, float *grad,
                        double *scal_out, int ctl_phase, cudaStream_t s)
{
    const Level &L = c->L[level];
    LevelGeom g = L.geom();
    int nD = 0;
    cudaError_t e;
    const bool fused = use_fused(c, level);
    const bool curv_in_pass = fused && fused_curv_in_pass(c, level);
    // The curvature Laplacian (node pass, HBM-light) runs on the side stream
    // beside the NGF pass (issue-bound, one CTA per SM), in the tail of its last
    // wave: fork before, join before the gradient assembly.  Captured, the two
    // become parallel graph branches.  With the batched form's arithmetic the
    // fused pass forms it itself, with one S partial per tile.
    e = cudaEventRecord(c->ev_fork, s);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    if (e != cudaSuccess)
        return e;
    if (c->time_ngf)
        e = cudaEventRecord(c->kev[0], s);
    if (e == cudaSuccess) {
        if (fused)
            e = launch_ngf_fused(c, level, ub, dir, t_dev, grad, c->es.partials, &nD, s);
        else
            e = launch_ngf_multipass(c, level, ub, dir, t_dev, grad, c->es.partials, &nD, s);
    }
    if (e == cudaSuccess && c->time_ngf)
        e = cudaEventRecord(c->kev[1], s);
    if (e != cudaSuccess)
        return e;
    dim3 blk(32, 8, 1);
    dim3 gn((L.n[0] + 31) / 32, (L.n[1] + 7) / 8, L.n[2]);
    dim3 gw(gn.x, gn.y, curv_zchunks(L.n[2]));
    double *pS = c->es.partials + nD;
    if (!curv_in_pass) {
        k_curv_w<<<gw, blk, 0, c->side>>>(g, ub, dir, t_dev, c->es.w, pS);
        c->launches += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaEventRecord(c->ev_join, c->side);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(s, c->ev_join, 0);
    if (e != cudaSuccess)
        return e;
    double hy = L.H[0] * L.H[1] * L.H[2];
    int nS = curv_in_pass ? nD : (int)(gw.x * gw.y * gw.z);
    // grad = (tile partials of P^T r) + alpha hbar_y L^T w, and J, D, S (+ control).  The
    // final reduction reads only the block partials of the kernels before, not the
    // gradient.  On small grids block 0 of the gather runs it first (one launch); on
    // large ones it is a one-block kernel on the side stream beside the gather, since
    // the control code in the gather would cost the large grid occupancy.
    if (fused && gather_blocks(L.n) < GATHER_SPLIT_BLOCKS)
        return launch_gather_fin(c, level, c->es.w, (float)(c->cfg.alpha * hy), grad, nD, pS, nS, scal_out,
                                 ctl_phase, s);
    if (fused) {
        const double hbar = L.h[0] * L.h[1] * L.h[2];
        e = cudaEventRecord(c->ev_fork, s);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
        if (e == cudaSuccess) {
            if (ctl_phase >= 0) {
                e = launch_finalize_ctl(c, c->es.partials, nD, pS, nS, 0.5 * hbar, c->cfg.alpha, 0.5 * hy, scal_out,
                                        ctl_phase, c->side);
            } else {
                k_finalize<<<1, 512, 0, c->side>>>(c->es.partials, nD, pS, nS, 0.5 * hbar, c->cfg.alpha, 0.5 * hy,
                                                    scal_out);
                e = cudaGetLastError();
            }
            c->launches += 1;
        }
        if (e == cudaSuccess)
            e = launch_gather_grad(c, level, c->es.w, (float)(c->cfg.alpha * hy), grad, s);
        if (e == cudaSuccess)
            e = cudaEventRecord(c->ev_join, c->side);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(s, c->ev_join, 0);
        return e;
    }
    // multi-pass: grad += alpha hbar_y L^T w, then the final reduction
    k_curv_grad<<<gn, blk, 0, s>>>(g, c->es.w, (float)(c->cfg.alpha * hy), grad);
    double hbar = L.h[0] * L.h[1] * L.h[2];
    c->launches += 2;
    if (ctl_phase >= 0)   // the reduction block also takes the line-search decision
        return launch_finalize_ctl(c, c->es.partials, nD, pS, nS, 0.5 * hbar, c->cfg.alpha, 0.5 * hy, scal_out,
                                   ctl_phase, s);
    k_finalize<<<1, 512, 0, s>>>(c->es.partials, nD, pS, nS, 0.5 * hbar, c->cfg.alpha, 0.5 * hy, scal_out);
    return cudaGetLastError();
}

// Partial-sum slots one evaluation at this level needs (fused or multi-pass).
int eval_partials_needed(const Level &L)
{
    long long vox_blocks = (long long)((L.m[0] + 31) / 32) * ((L.m[1] + 7) / 8) * L.m[2];
    long long node_blocks = (long long)((L.n[0] + 31) / 32) * ((L.n[1] + 7) / 8) * L.n[2];
    return (int)(vox_blocks + node_blocks + 1024);
}

// Explicit-buffer launch of the final reduction, for callers that own every
// buffer (the allocation-free entry point).

cudaError_t launch_finalize_raw(const double *pD, int nD, const double *pS, int nS, double hbar_half, double alpha,
                                double hy_half, double *scal, cudaStream_t s)
{
    k_finalize<<<1, 512, 0, s>>>(pD, nD, pS, nS, hbar_half, alpha, hy_half, scal);
    return cudaGetLastError();
}
