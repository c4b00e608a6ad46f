// FP64 control of the device-resident L-BFGS (Sec. 2.1: L-BFGS of Nocedal
// 1980 with Armijo backtracking): the scalar decisions of every phase, run by
// one block - the block that completes the cross-block reduction of the kernel
// before them, or a control kernel of the batched form.  Shared by the
// translation units whose kernels take a control phase.
#pragma once

#include <math.h>

#include "internal.h"

namespace {

constexpr int CT = 256;             // threads of the control kernel (the phase needs at most this many)
constexpr int ND_ACC = 2 + 4 * LB_MAXS;

__device__ void set_p0(LbfgsState *st)
{
    st->dcount = 0;
    st->cg = st->ginf > 0.0 ? -st->Hmin / st->ginf : 0.0;
}

// Compact form: with R = upper triangle of S'Y (by age), D its diagonal,
// gamma = s'y / y'y of the newest pair, q = R^{-1} S'g and
// w = R^{-T} ((D + gamma Y'Y) q - gamma Y'g):
//   H g = gamma g + S w - gamma Y q,   p = -H g.
// Run by one full warp, lane i holding row i: the triangular solves go column
// by column (q_i, then every remaining row updated at once), so the FP64
// dependency chain is about 3 count operations long.  1 / R_ii and gamma are
// taken once, when the pair is stored (FP64 divides cost ~640 cycles here).
__device__ void set_compact_warp(LbfgsState *st)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = linear_tid() & 31;
    const int c = st->count;
    const bool row = lane < c;
    const int oi = row ? st->order[lane] : 0;
    const double gamma = st->gamma;
    const double Rii = row ? st->SY[oi][oi] : 0.0;
    const double iR = row ? st->iSY[oi] : 0.0;
    const double Yg = row ? st->Yg[oi] : 0.0;
    double r = row ? st->tscale[oi] * st->Pg[oi] : 0.0;   // S'g
    double q = 0.0;
    for (int i = c - 1; i >= 0; i--) {   // R q = S'g, upper triangular
        const double qi = __shfl_sync(FULL, r * iR, i);
        if (lane == i)
            q = qi;
        if (lane < i)
            r = fma(-st->SY[oi][st->order[i]], qi, r);
    }
    double acc = 0.0;                     // (Y'Y q)_i
    for (int j = 0; j < c; j++) {
        const double qj = __shfl_sync(FULL, q, j);
        if (row)
            acc = fma(st->YY[oi][st->order[j]], qj, acc);
    }
    r = fma(Rii, q, gamma * (acc - Yg));  // (D + gamma Y'Y) q - gamma Y'g
    double w = 0.0;
    for (int i = 0; i < c; i++) {        // R^T w = r, lower triangular
        const double wi = __shfl_sync(FULL, r * iR, i);
        if (lane == i)
            w = wi;
        if (lane > i && row)
            r = fma(-st->SY[st->order[i]][oi], wi, r);
    }
    if (lane == 0) {
        st->dcount = c;
        st->cg = -gamma;
    }
    if (row) {
        st->dslot[lane] = oi;
        st->cp[lane] = -w * st->tscale[oi];
        st->cy[lane] = gamma * q;
    }
}

__device__ bool finite_d(double x) { return isfinite(x); }

// One entry of a block's partials as a double-float: an FP32 block partial
// (grids of at most LB_DIRECT blocks) or a double-float group sum.
__device__ __forceinline__ DFloat df_load(const float *__restrict__ x, long long i)
{
    return DFloat{__ldcg(x + i), 0.f};
}
__device__ __forceinline__ DFloat df_load(const float2 *__restrict__ x, long long i)
{
    const float2 v = __ldcg(x + i);
    return DFloat{v.x, v.y};
}

// Ordered double-float sum of count entries x[i0], x[i0 + step], ... (is_max:
// their maximum; the max entries are maxima of FP32 absolute values, exact in
// hi).  The loads go out 8 at a time so that their L2 round trips overlap; the
// additions keep the index order.
template <typename T>
__device__ __forceinline__ DFloat df_ordered_reduce(const T *__restrict__ x, long long i0, int count, long long step,
                                                    bool is_max)
{
    DFloat s{0.f, 0.f};
    for (int k0 = 0; k0 < count; k0 += 8) {
        DFloat v[8];
#pragma unroll
        for (int k = 0; k < 8; k++)
            v[k] = k0 + k < count ? df_load(x, i0 + (long long)(k0 + k) * step) : DFloat{0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 8; k++)
            if (k0 + k < count)
                s = is_max ? DFloat{fmaxf(s.hi, v[k].hi), 0.f} : df_add(s, v[k]);
    }
    return s;
}

// Cross-block sum (entry imax: max) of nd values over nparts partials
// (partials[b * nd + d]) in a fixed order, as double-float: thread (d, j)
// sums partials j, j + J, ... for J groups per value (J about sqrt(nparts),
// at most CT / nd), then thread d adds its J group sums and rounds the pair
// to FP64 in red[d].
template <typename T>
__device__ __forceinline__ void control_reduce(const T *__restrict__ partials, int nparts, int nd, int imax,
                                               double *red, DFloat *scratch)
{
    const int t = linear_tid();
    int J = 1;
    while (J * J < nparts)
        J++;
    if (J > CT / nd)
        J = CT / nd;
    if (t < nd * J) {
        const int d = t % nd, j = t / nd;
        const int count = j < nparts ? (nparts - j + J - 1) / J : 0;
        scratch[t] = df_ordered_reduce(partials, (long long)j * nd + d, count, (long long)J * nd, d == imax);
    }
    __syncthreads();
    if (t < nd) {
        DFloat s = scratch[t];
        for (int j = 1; j < J; j++) {
            const DFloat x = scratch[j * nd + t];
            s = (t == imax) ? DFloat{fmaxf(s.hi, x.hi), 0.f} : df_add(s, x);
        }
        red[t] = df_to_double(s);
    }
    __syncthreads();
}

// The control state in shared memory, one copy per block: the single decision
// thread works on it there (one coalesced copy in and out instead of hundreds
// of dependent global accesses).  A vector pass loads it when it starts, so the
// block that ends up running the control does not wait for it.
constexpr int STATE_WORDS = (int)(sizeof(LbfgsState) / sizeof(int));

__device__ __forceinline__ LbfgsState &ctl_state()
{
    __shared__ LbfgsState S;
    return S;
}

// every thread of the block; the caller synchronises before reading
__device__ __forceinline__ void ctl_state_load(const LbfgsState *gst)
{
    int *dst = reinterpret_cast<int *>(&ctl_state());
    const int *src = reinterpret_cast<const int *>(gst);
    for (int i = linear_tid(); i < STATE_WORDS; i += nthreads())
        dst[i] = __ldcg(src + i);   // through L2: other blocks' control phases write it within a launch
}

// Fence of one thread after a block barrier: with the barrier it orders the
// block's earlier writes before the arrival that follows (release), or the
// other blocks' writes before the block's reads (acquire).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// The phase's sums come from FP32 block partials pf or double-float group sums
// pg (nparts of either; both null for the phases that reduce nothing).
// preloaded: ctl_state() already holds gst (ctl_state_load at the kernel's start)
__device__ __forceinline__ void lb_control_body(int phase, LbfgsState *gst, const float *__restrict__ pf,
                                                    const float2 *__restrict__ pg, int nparts,
                                                    const double *__restrict__ scal, unsigned long long h_ls,
                                                    unsigned long long h_iter, unsigned long long h_redo,
                                                    bool preloaded = false)
{
    __shared__ double red[ND_ACC];
    __shared__ DFloat scratch[CT];
    __shared__ int s_store, s_compact;
    constexpr int NW = STATE_WORDS;
    LbfgsState &S = ctl_state();
    if (!preloaded)
        ctl_state_load(gst);
    else if (linear_tid() == 0)   // set by another block of this pass after the preload
        S.wait_err = *reinterpret_cast<volatile const int *>(&gst->wait_err);
    __syncthreads();
    LbfgsState *st = &S;
    const int nd = phase == LB_ACCEPTED ? ND_ACC : 2;
    const int imax = (phase == LB_INIT || phase == LB_ACCEPTED) ? 1 : -1;
    const bool need = phase != LB_ARMIJO && !(phase == LB_ACCEPTED && (!st->active || st->ls != LS_ACCEPTED)) &&
                      !(phase == LB_DIR_REDO && !st->redo_dir) && !(phase == LB_DIR && !st->iter_continue);
    if (need && pf)
        control_reduce(pf, nparts, nd, imax, red, scratch);
    else if (need && pg)
        control_reduce(pg, nparts, nd, imax, red, scratch);
    __syncthreads();
    if (linear_tid() == 0) {
    s_store = 0;
    s_compact = 0;
    switch (phase) {
    case LB_INIT: {
        st->J = __ldcg(scal);   // the objective's scalars, through L2 (written within a launch)
        st->D = __ldcg(scal + 1);
        st->S = __ldcg(scal + 2);
        st->J0 = st->J;
        st->gg = red[0];
        st->ginf = red[1];
        st->g0norm = sqrt(red[0]);
        st->gtol2 = st->tol_grad_rel * st->tol_grad_rel * red[0];
        st->k = 0;
        st->bodies = 0;
        st->evals = 1;
        st->small_count = 0;
        st->count = 0;
        st->free_slot = 0;
        st->status = 0;
        st->retried = 0;
        st->redo_dir = 0;
        st->redos = 0;
        st->done = 0;
        if (!finite_d(st->J) || !finite_d(st->gg)) {
            st->status = -5;
            st->done = 1;
        }
        if (st->max_iter <= 0 || st->g0norm == 0.0)
            st->done = 1;
        set_p0(st);
        st->iter_continue = !st->done;
        st->active = 0;
        st->ls_continue = 0;
        break;
    }
    case LB_DIR: {
        st->active = st->iter_continue;
        if (!st->iter_continue)
            break;
        st->gtp = red[0];
        st->pp = red[1];
        st->redo_dir = 0;
        if (!(st->gtp < 0.0) && st->dcount > 0) { // not a descent direction: reset the memory
            st->count = 0;
            set_p0(st);
            st->redo_dir = 1;
            st->redos++;
        }
        st->t = 1.0;
        st->trial = 0;
        st->ls = LS_RUNNING;
        st->ls_continue = 1;
        break;
    }
    case LB_DIR_REDO: {
        if (!st->redo_dir)
            break;
        st->gtp = red[0];
        st->pp = red[1];
        st->redo_dir = 0;
        break;
    }
    case LB_ARMIJO: {
        if (!st->active || !st->ls_continue)   // this pair is not searching (batched levels)
            break;
        st->Jt = __ldcg(scal);
        st->Dt = __ldcg(scal + 1);
        st->St = __ldcg(scal + 2);
        st->evals++;
        if (finite_d(st->Jt) && st->Jt <= st->J + st->c1 * st->t * st->gtp) {
            st->ls = LS_ACCEPTED;
            st->ls_continue = 0;
            st->lcount = st->count + 1;
            for (int j = 0; j < st->count; j++)
                st->lslot[j] = st->order[j];
            st->lslot[st->count] = st->free_slot;
        } else {
            st->trial++;
            if (st->trial >= st->max_bt) {
                st->ls_continue = 0;
                if (st->dcount > 0 && !st->retried) { // one retry from a fresh memory
                    st->ls = LS_RETRY;
                    st->retried = 1;
                    st->count = 0;
                    set_p0(st);
                } else {
                    st->ls = LS_FAILED;
                    st->status = 1;
                    st->done = 1;
                }
            } else {
                st->t *= 0.5;
            }
        }
        break;
    }
    case LB_ACCEPTED: {
        if (!st->active)   // this pair did not run the iteration (batched levels)
            break;
        if (++st->bodies > 2 * st->max_iter + 8) {   // cannot happen with the rules below; a hard stop
            st->status = -6;
            st->done = 1;
            st->iter_continue = 0;
            break;
        }
        if (st->ls == LS_RETRY) {
            st->iter_continue = 1;
            break;
        }
        if (st->ls != LS_ACCEPTED) {
            st->iter_continue = 0;
            break;
        }
        for (int j = 0; j < st->lcount; j++) {
            int s = st->lslot[j];
            st->Pg[s] = red[2 + 4 * j];
            st->Yg[s] = red[3 + 4 * j];
            st->Py[s] = red[4 + 4 * j];
            st->Yy[s] = red[5 + 4 * j];
        }
        double Jprev = st->J;
        st->J = st->Jt;
        st->D = st->Dt;
        st->S = st->St;
        st->k++;
        st->gg = red[0];
        st->ginf = red[1];
        const int f = st->free_slot;
        const double tn = st->t;
        double sy = tn * st->Py[f], ss = tn * tn * st->pp, yy = st->Yy[f];
        // curvature test s'y > 1e-10 ||s|| ||y||, compared as squares (sy > 0)
        if (sy > 0.0 && sy * sy > 1e-20 * ss * yy) {   // keep the pair
            st->tscale[f] = tn;
            s_store = 1;   // 1 / s'y and gamma are formed by the warp below
            for (int j = 0; j < st->lcount; j++) {
                int s = st->lslot[j];
                st->SY[s][f] = st->tscale[s] * st->Py[s];
                st->YY[s][f] = st->Yy[s];
                st->YY[f][s] = st->Yy[s];
            }
            if (st->count == st->m) {
                int ev = st->order[0];
                for (int j = 0; j < st->m - 1; j++)
                    st->order[j] = st->order[j + 1];
                st->order[st->m - 1] = f;
                st->free_slot = ev;
            } else {
                st->order[st->count++] = f;
                unsigned used = 0;
                for (int j = 0; j < st->count; j++)
                    used |= 1u << st->order[j];
                int fs = 0;
                while (used & (1u << fs))
                    fs++;
                st->free_slot = fs;
            }
        }
        st->retried = 0;
        if (!finite_d(st->J) || !finite_d(st->gg)) {
            st->status = -5;
            st->done = 1;
        } else if (st->k >= st->max_iter) {
            st->done = 1;
        } else if (!st->fixed_iters) {
            if (st->gg <= st->gtol2) {   // ||g|| <= tol_grad_rel ||g0||
                st->done = 1;
            } else if (fabs(Jprev - st->J) <= st->tol_j_rel * (1.0 + fabs(st->J0))) {
                if (++st->small_count >= st->tol_j_count)
                    st->done = 1;
            } else {
                st->small_count = 0;
            }
        }
        if (!st->done) {
            if (st->count > 0)
                s_compact = 1;
            else
                set_p0(st);
        }
        st->iter_continue = !st->done;
        break;
    }
    default:
        break;
    }
    if (st->wait_err) {   // a vector pass lost chunks: its sums are incomplete, stop the level
        st->wait_err = 0;
        st->test_drop = 0;
        st->status = -7;
        st->done = 1;
        st->iter_continue = 0;
        st->ls_continue = 0;
        st->redo_dir = 0;
        s_store = 0;
        s_compact = 0;
    }
    }   // thread 0
    __syncthreads();
    if (linear_tid() < 32 && (s_store || s_compact)) {
        const int lane = linear_tid();
        if (s_store) {   // the pair in the free slot's predecessor position was stored
            const int f = st->order[st->count - 1];
            const double num = lane == 1 ? st->SY[f][f] : 1.0;
            const double den = lane == 1 ? st->YY[f][f] : st->SY[f][f];
            const double x = num / den;   // lanes 0 and 1 divide at once
            const double gm = __shfl_sync(0xffffffffu, x, 1);
            if (lane == 0) {
                st->iSY[f] = x;
                st->gamma = gm;
            }
            __syncwarp();
        }
        if (s_compact)
            set_compact_warp(st);
    }
#if CUDART_VERSION >= 12040
    if (linear_tid() == 0) {
        if (h_ls)
            cudaGraphSetConditional((cudaGraphConditionalHandle)h_ls, st->ls_continue ? 1u : 0u);
        if (h_iter)
            cudaGraphSetConditional((cudaGraphConditionalHandle)h_iter, st->iter_continue ? 1u : 0u);
        if (h_redo)
            cudaGraphSetConditional((cudaGraphConditionalHandle)h_redo, st->redo_dir ? 1u : 0u);
    }
#endif
    __syncthreads();
    for (int i = linear_tid(); i < NW; i += nthreads())
        reinterpret_cast<int *>(gst)[i] = reinterpret_cast<const int *>(&S)[i];
}

}  // namespace
