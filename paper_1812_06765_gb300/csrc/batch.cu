// Batched registration of many pairs of uneven size (reg_register_batch).
//
// Per pyramid level, all pairs run their L-BFGS iterations in lock step inside
// one CUDA graph: every kernel of an iteration is launched once for the whole
// batch and walks a work list of (pair, item) over all pairs - fused-pass
// tiles, node blocks, vector blocks - with a persistent grid.  Each item runs
// the same per-pair code as a single registration with that pair's own
// buffers, tiling and block counts, so every pair gets exactly the result it
// gets alone.  Pairs that have finished their level, or their line search,
// skip their items; the loops run while any pair still iterates / searches.
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <vector>

#include "batch.h"

namespace {

long long ring_stride(long long n) { return (n + 3) & ~3LL; }

void fill_pair_level(reg_ctx *c, int level, PairLevel &P)
{
    const Level &L = c->L[level];
    P = PairLevel{};
    P.geom = L.geom();
    FusedSplit split;
    int ntx, nty;
    fused_tiling(L, c->num_sms, &split, &ntx, &nty);
    const bool bf16 = c->cfg.image_dtype == 1 && L.Tb && L.Rb;
    FusedArgs a{};
    a.g = P.geom;
    a.T = bf16 ? static_cast<const void *>(L.Tb) : static_cast<const void *>(L.Tp);   // zero-bordered copies
    a.R = bf16 ? static_cast<const void *>(L.Rb) : static_cast<const void *>(L.R);
    a.Rn = bf16 ? nullptr : L.Rn;   // R's normalized gradient field (FP32 images)
    a.ub = c->lb.u;
    a.dir = nullptr;
    a.t_dev = nullptr;
    a.tau = (float)c->cfg.tau;
    a.rho = (float)c->cfg.rho;
    a.split = split;
    a.ntx = ntx;
    a.nty = nty;
    a.part = c->es.part;
    a.partials = c->es.partials;
    a.w = c->es.w;
    a.partials_S = c->es.partials + ntx * nty * split.count();   // after the D partials
    P.fa_init = a;
    a.dir = c->lb.pdir;
    a.t_dev = &c->lb.st->t;
    P.fa_trial = a;
    P.ntx = ntx;
    P.nty = nty;
    P.gbx = gather_runs_per_plane(L.n);
    P.nD = ntx * nty * split.count();
    P.nS = P.nD;   // the fused pass writes one S partial per tile
    P.ngather = P.gbx * L.n[2];
    P.w = c->es.w;
    P.pS = c->es.partials + P.nD;
    const double hy = L.H[0] * L.H[1] * L.H[2];
    P.hbar_half = 0.5 * L.h[0] * L.h[1] * L.h[2];
    P.alpha = c->cfg.alpha;
    P.hy_half = 0.5 * hy;
    P.alpha_hy = (float)(c->cfg.alpha * hy);
    P.scal = c->es.scal;
    P.scal_t = c->lb.scal_t;
    P.st = c->lb.st;
    P.n = 3 * L.nn;
    P.stride = ring_stride(P.n);
    P.u = c->lb.u;
    P.g = c->lb.g;
    P.gt = c->lb.gt;
    P.pdir = c->lb.pdir;
    P.P = c->lb.P;
    P.Y = c->lb.Y;
    P.lpart = c->lb.partials;
    P.lgpart = c->lb.gpart;
    P.lcnt = c->lb.cnt;
    P.nchunks = num_blocks_for(c, (P.n + 3) / 4, LB_VT);
}

struct BatchDev {
    PairLevel *pl = nullptr;
    int *off = nullptr;      // [3][npairs + 1]: tiles, gather blocks, vector blocks
    int *counters = nullptr; // [4]: runs of the iteration and search conditions, then their last values
};

struct CaptureGuard {
    cudaStream_t s;
    bool active = false;
    ~CaptureGuard()
    {
        if (active) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(s, &g);
            if (g)
                cudaGraphDestroy(g);
        }
    }
};

cudaError_t leaves_of(cudaStream_t s, std::vector<cudaGraphNode_t> &out)
{
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &nd);
    if (e == cudaSuccess)
        out.assign(deps, deps + nd);
    return e;
}

cudaError_t while_node(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps, cudaGraphConditionalHandle h,
                       cudaGraphNode_t *node, cudaGraph_t *body)
{
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaError_t e = cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p);
    if (e == cudaSuccess)
        *body = p.conditional.phGraph_out[0];
    return e;
}

struct BatchLaunch {
    const BatchDev *d;
    int npairs, tiles, nodes, chunks;
    int g_fused, g_nodes, g_chunks;
    bool bf16;
    int device;

    cudaError_t eval(int mode, cudaStream_t s) const
    {
        // the fused pass also forms each pair's curvature Laplacian and S partials
        cudaError_t e = launch_fused_batch(d->pl, d->off, npairs, tiles, mode, bf16, g_fused, device, s);
        if (e == cudaSuccess)
            e = launch_gather_batch(d->pl, d->off + (npairs + 1), npairs, nodes, mode, g_nodes, s);
        if (e == cudaSuccess)
            e = launch_finalize_batch(d->pl, npairs, mode, s);
        return e;
    }
    cudaError_t vec(int step, cudaStream_t s) const
    {
        return launch_lb_vector_batch(d->pl, d->off + 2 * (npairs + 1), npairs, chunks, step, g_chunks, s);
    }
    cudaError_t ctl(int phase, cudaStream_t s) const { return launch_lb_control_batch(d->pl, npairs, phase, s); }
    cudaError_t cond(int which, cudaGraphConditionalHandle h, cudaStream_t s) const
    {
        return launch_batch_condition(d->pl, npairs, which, h, d->counters, s);
    }
};

#define BK(call)                                  \
    do {                                          \
        cudaError_t _e = (call);                  \
        if (_e != cudaSuccess) {                  \
            if (G) cudaGraphDestroy(G);           \
            return _e;                            \
        }                                         \
    } while (0)

// The whole level for all pairs: init, then WHILE any pair iterates
// { direction; WHILE any pair searches { objective at the trial points; Armijo }; accept }.
cudaError_t build_batch_graph(const BatchLaunch &B, cudaStream_t cs, cudaGraphExec_t *out)
{
    cudaGraph_t G = nullptr;
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    BK(cudaGraphCreate(&G, 0));
    cudaGraphConditionalHandle h_iter, h_ls;
    BK(cudaGraphConditionalHandleCreate(&h_iter, G, 0, cudaGraphCondAssignDefault));
    std::vector<cudaGraphNode_t> leaves;
    cudaGraph_t g2 = nullptr;
    {
        CaptureGuard guard{cs};
        BK(cudaStreamBeginCaptureToGraph(cs, G, nullptr, nullptr, 0, mode));
        guard.active = true;
        BK(B.eval(0, cs));
        BK(B.vec(0, cs));
        BK(B.ctl(LB_INIT, cs));
        BK(B.cond(0, h_iter, cs));
        BK(leaves_of(cs, leaves));
        guard.active = false;
        BK(cudaStreamEndCapture(cs, &g2));
    }
    cudaGraphNode_t w_iter, w_ls;
    cudaGraph_t body = nullptr, ls_body = nullptr;
    BK(while_node(G, leaves, h_iter, &w_iter, &body));
    BK(cudaGraphConditionalHandleCreate(&h_ls, body, 0, cudaGraphCondAssignDefault));
    {
        CaptureGuard guard{cs};
        BK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, mode));
        guard.active = true;
        BK(B.vec(1, cs));
        BK(B.ctl(LB_DIR, cs));
        BK(B.vec(2, cs));
        BK(B.ctl(LB_DIR_REDO, cs));
        BK(B.cond(1, h_ls, cs));
        BK(leaves_of(cs, leaves));
        guard.active = false;
        BK(cudaStreamEndCapture(cs, &g2));
    }
    BK(while_node(body, leaves, h_ls, &w_ls, &ls_body));
    {
        CaptureGuard guard{cs};
        BK(cudaStreamBeginCaptureToGraph(cs, ls_body, nullptr, nullptr, 0, mode));
        guard.active = true;
        BK(B.eval(1, cs));
        BK(B.ctl(LB_ARMIJO, cs));
        BK(B.cond(1, h_ls, cs));
        guard.active = false;
        BK(cudaStreamEndCapture(cs, &g2));
    }
    {
        CaptureGuard guard{cs};
        BK(cudaStreamBeginCaptureToGraph(cs, body, &w_ls, nullptr, 1, mode));
        guard.active = true;
        BK(B.vec(3, cs));
        BK(B.ctl(LB_ACCEPTED, cs));
        BK(B.cond(0, h_iter, cs));
        guard.active = false;
        BK(cudaStreamEndCapture(cs, &g2));
    }
    BK(cudaGraphInstantiate(out, G, 0));
    cudaGraphDestroy(G);
    return cudaSuccess;
}

int cap(long long v, long long hi) { return (int)(v < 1 ? 1 : (v > hi ? hi : v)); }

// Tiling rules of a batched level: 0 each pair's own split (its single-pair
// autotuning), -1 the throughput rule (fewest z steps in total), T > 0 equal
// segments of T planes for every pair (halved while a segment would span the
// pair's depth twice).
FusedSplit rule_split(int rule, const Level &L, const FusedSplit &own)
{
    if (rule == 0 && own.valid())
        return own;
    if (rule <= 0)
        return fused_split_uniform(fused_tz_throughput(L), L.m[2]);
    int tz = rule;
    while (tz > 2 && tz / 2 >= L.m[2])
        tz /= 2;
    return fused_split_uniform(tz, L.m[2]);
}

std::mutex g_btune_mu;
std::map<std::vector<int>, int> g_btune;   // (level, SMs, image type, pair dims...) -> rule

// Batch autotuner: times the batched fused pass (at the pairs' current u) under
// each candidate rule - one warm launch, then the better of two event timings -
// and returns the fastest rule.  Cached per batch geometry for the process.
int batch_tiling_rule(reg_handle *hs, int n, int l, const std::vector<FusedSplit> &own, BatchDev &d,
                      std::vector<PairLevel> &hpl, std::vector<int> &hoff, bool bf16, cudaStream_t s,
                      cudaError_t *err)
{
    reg_ctx *c0 = hs[0];
    std::vector<int> key{l, c0->num_sms, bf16 ? 1 : 0};
    for (int i = 0; i < n; i++)
        for (int k = 0; k < 3; k++)
            key.push_back(hs[i]->L[l].m[k]);
    {
        std::lock_guard<std::mutex> lk(g_btune_mu);
        auto it = g_btune.find(key);
        if (it != g_btune.end())
            return it->second;
    }
    static const int rules[] = {0, -1, 16, 32, 64, 128};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    int best = -1;
    float best_ms = 0.f;
    for (int rule : rules) {
        if (e != cudaSuccess)
            break;
        int tiles = 0;
        for (int i = 0; i < n; i++) {
            hs[i]->L[l].split = rule_split(rule, hs[i]->L[l], own[i]);
            fill_pair_level(hs[i], l, hpl[i]);
            hoff[i] = tiles;
            tiles += hpl[i].nD;
        }
        hoff[n] = tiles;
        e = cudaMemcpyAsync(d.pl, hpl.data(), sizeof(PairLevel) * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d.off, hoff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s);
        float t = 0.f;
        for (int r = -1; r < 2 && e == cudaSuccess; r++) {
            if (r >= 0)
                e = cudaEventRecord(e0, s);
            if (e == cudaSuccess)
                e = launch_fused_batch(d.pl, d.off, n, tiles, 0, bf16, cap(tiles, (long long)fused_slots(c0->num_sms)), c0->device, s);
            if (e == cudaSuccess && r >= 0)
                e = cudaEventRecord(e1, s);
            if (e == cudaSuccess && r >= 0)
                e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess && r >= 0)
                e = cudaEventElapsedTime(&ms, e0, e1);
            if (r >= 0)
                t = (r == 0 || ms < t) ? ms : t;
        }
        if (e == cudaSuccess && (best == -1 || t < best_ms)) {
            best = rule;
            best_ms = t;
        }
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    *err = e;
    if (e != cudaSuccess)
        return -1;
    std::lock_guard<std::mutex> lk(g_btune_mu);
    g_btune[key] = best;
    return best;
}

// The same level, queued from the host (use_graph = 0): the kernels of the graph
// in the same order, the loop conditions read back after each condition kernel.
// For profilers that cannot see the kernels inside conditional graph nodes.
cudaError_t run_batch_level_host(const BatchLaunch &B, int *counters, cudaStream_t s, int max_rounds)
{
    int h[4];
    auto cond = [&](int which, bool &out) -> cudaError_t {
        cudaError_t e = B.cond(which, 0, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h, counters, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        out = h[2 + which] != 0;
        return e;
    };
#define HK(call)                             \
    do {                                     \
        cudaError_t _e = (call);             \
        if (_e != cudaSuccess) return _e;    \
    } while (0)
    bool it = false, ls = false;
    HK(B.eval(0, s));
    HK(B.vec(0, s));
    HK(B.ctl(LB_INIT, s));
    HK(cond(0, it));
    int rounds = 0;   // bounded like the graph: every pair stops after its own bounded loops
    while (it && rounds++ < max_rounds) {
        HK(B.vec(1, s));
        HK(B.ctl(LB_DIR, s));
        HK(B.vec(2, s));
        HK(B.ctl(LB_DIR_REDO, s));
        HK(cond(1, ls));
        while (ls && rounds++ < max_rounds) {
            HK(B.eval(1, s));
            HK(B.ctl(LB_ARMIJO, s));
            HK(cond(1, ls));
        }
        HK(B.vec(3, s));
        HK(B.ctl(LB_ACCEPTED, s));
        HK(cond(0, it));
    }
#undef HK
    return rounds > max_rounds ? cudaErrorTimeout : cudaSuccess;
}

}  // namespace

extern "C" int reg_register_batch(reg_handle *hs, int n, float **u_out, int out_is_device, reg_stats *stats)
{
    if (!hs || n < 1 || !u_out)
        return set_err(nullptr, REG_ERR_ARG, "reg_register_batch: NULL argument or n < 1");
    reg_ctx *c0 = hs[0];
    for (int i = 0; i < n; i++) {
        reg_ctx *c = hs[i];
        if (!c || !u_out[i])
            return set_err(nullptr, REG_ERR_ARG, "reg_register_batch: NULL handle or output %d", i);
        if (!c->have_images)
            return set_err(nullptr, REG_ERR_STATE, "reg_register_batch: pair %d has no images", i);
        if (c->levels != c0->levels || c->cfg.image_dtype != c0->cfg.image_dtype || c->device != c0->device ||
            (c->cfg.start_level < 0 ? c->levels - 1 : c->cfg.start_level) !=
                (c0->cfg.start_level < 0 ? c0->levels - 1 : c0->cfg.start_level))
            return set_err(nullptr, REG_ERR_ARG,
                           "reg_register_batch: pairs must share levels, start level, image type and device (pair %d)", i);
        for (int l = 0; l < c->levels; l++)
            if (!use_fused(c, l))
                return set_err(nullptr, REG_ERR_ARG,
                               "reg_register_batch: pair %d level %d is not a ratio-2 grid (even dims, default "
                               "node counts, eval_impl 0)", i, l);
        for (int j = 0; j < i; j++)
            if (hs[j] == c)
                return set_err(nullptr, REG_ERR_ARG, "reg_register_batch: handle %d repeats handle %d", i, j);
    }
    cudaStream_t s = c0->stream;
    reg_ctx *c = c0;   // for CK
    const int levels = c0->levels;
    const int start = c0->cfg.start_level < 0 ? levels - 1 : c0->cfg.start_level;
    const bool bf16 = c0->cfg.image_dtype == 1;
    std::vector<reg_stats> st(n);
    for (int i = 0; i < n; i++) {
        memset(&st[i], 0, sizeof(reg_stats));
        st[i].levels = levels;
    }
    BatchDev d;
    CK(cudaMallocAsync((void **)&d.pl, sizeof(PairLevel) * n, s));
    CK(cudaMallocAsync((void **)&d.off, sizeof(int) * 3 * (n + 1), s));
    CK(cudaMallocAsync((void **)&d.counters, sizeof(int) * 4, s));
    // every pair's own stream work (prolongations, state uploads) is ordered on c0's stream
    for (int i = 0; i < n; i++) {
        CK(cudaMemsetAsync(hs[i]->lb.u, 0, sizeof(float) * 3 * hs[i]->L[start].nn, s));
        CK(cudaMemsetAsync(hs[i]->lb.cnt, 0, sizeof(unsigned) * hs[i]->lb.cnt_len, s));
    }
    long long launches = 0;
    int status = REG_OK;
    std::vector<PairLevel> hpl(n);
    std::vector<int> hoff(3 * (n + 1));
    if (!c0->lev_ev[0])
        for (int i = 0; i <= REG_MAX_LEVELS; i++)
            CK(cudaEventCreate(&c0->lev_ev[i]));
    for (int l = start; l >= 0 && status >= 0; l--) {
        CK(cudaEventRecord(c0->lev_ev[l + 1], s));
        int tiles = 0, nodes = 0, chunks = 0;
        // Tiling of the batched level: the batch keeps every SM busy, so the
        // single-pair tiling of each handle is not necessarily the right one.
        // hs[0]'s cfg.fused_tz forces a rule; otherwise the batch autotuner picks
        // one (each handle's own tiling is restored after the level).
        std::vector<FusedSplit> own(n);
        for (int i = 0; i < n; i++)
            own[i] = hs[i]->L[l].split;
        struct RestoreSplit {
            reg_handle *hs;
            int n, l;
            std::vector<FusedSplit> &split;
            ~RestoreSplit()
            {
                for (int i = 0; i < n; i++)
                    hs[i]->L[l].split = split[i];
            }
        } restore{hs, n, l, own};
        if (l < start)   // u at the level start: prolonged from the coarser level
            for (int i = 0; i < n; i++) {
                reg_ctx *ci = hs[i];
                CK(launch_prolong(ci->L[l + 1], ci->L[l], ci->lb.u, ci->lb.g, s));
                CK(cudaMemcpyAsync(ci->lb.u, ci->lb.g, sizeof(float) * 3 * ci->L[l].nn, cudaMemcpyDeviceToDevice,
                                   s));
                launches++;
            }
        int rule = c0->cfg.fused_tz;
        if (rule == 0 && !c0->cfg.autotune)
            rule = -1;
        if (rule == 0) {   // timed at the pairs' u of the level start
            cudaError_t te = cudaSuccess;
            rule = batch_tiling_rule(hs, n, l, own, d, hpl, hoff, bf16, s, &te);
            CK(te);
        }
        for (int i = 0; i < n; i++)
            hs[i]->L[l].split = rule_split(rule, hs[i]->L[l], own[i]);
        for (int i = 0; i < n; i++)
            st[i].tiling[l] = rule;
        for (int i = 0; i < n; i++) {
            reg_ctx *ci = hs[i];
            const Level &L = ci->L[l];
            double Hmin = fmin(L.H[0], fmin(L.H[1], L.H[2]));
            lbfgs_state_reset_host(ci->lb.st_host, ci->cfg, ci->cfg.max_iter[l], Hmin);
            CK(cudaMemcpyAsync(ci->lb.st, ci->lb.st_host, sizeof(LbfgsState), cudaMemcpyHostToDevice, s));
            fill_pair_level(ci, l, hpl[i]);
            hoff[i] = tiles;
            hoff[(n + 1) + i] = nodes;
            hoff[2 * (n + 1) + i] = chunks;
            tiles += hpl[i].nD;
            nodes += hpl[i].ngather;
            chunks += hpl[i].nchunks;
        }
        hoff[n] = tiles;
        hoff[(n + 1) + n] = nodes;
        hoff[2 * (n + 1) + n] = chunks;
        CK(cudaMemcpyAsync(d.pl, hpl.data(), sizeof(PairLevel) * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d.off, hoff.data(), sizeof(int) * hoff.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(d.counters, 0, sizeof(int) * 4, s));
        BatchLaunch B{&d, n, tiles, nodes, chunks, cap(tiles, (long long)fused_slots(c0->num_sms)), cap(nodes, 8LL * c0->num_sms),
                      cap(chunks, 4LL * c0->num_sms), bf16, c0->device};
        cudaError_t e = cudaSuccess;
        if (c0->cfg.use_graph) {
            cudaGraphExec_t exec = nullptr;
            e = build_batch_graph(B, c0->cap_stream, &exec);
            if (e != cudaSuccess) {
                cudaFreeAsync(d.pl, s);
                cudaFreeAsync(d.off, s);
                cudaFreeAsync(d.counters, s);
                return cuda_err(c0, e, "reg_register_batch: building the level graph");
            }
            e = cudaGraphLaunch(exec, s);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(s);
            cudaGraphExecDestroy(exec);
        } else {
            int max_it = 0, max_bt = 0;
            for (int i = 0; i < n; i++) {
                max_it = max_it > hs[i]->cfg.max_iter[l] ? max_it : hs[i]->cfg.max_iter[l];
                max_bt = max_bt > hs[i]->cfg.max_backtracks ? max_bt : hs[i]->cfg.max_backtracks;
            }
            e = run_batch_level_host(B, d.counters, s, 4 * (max_it + 1) * (max_bt + 1) + 16);
        }
        int cnt[2] = {0, 0};
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cnt, d.counters, sizeof cnt, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        CK(e);
        // launches: init 7; per iteration body 8; per search round 6
        const long long bodies = cnt[0] - 1, rounds = cnt[1] - bodies;
        launches += 7 + 8 * bodies + 6 * rounds;
        for (int i = 0; i < n; i++) {
            reg_ctx *ci = hs[i];
            CK(cudaMemcpyAsync(ci->lb.st_host, ci->lb.st, sizeof(LbfgsState), cudaMemcpyDeviceToHost, s));
        }
        CK(cudaStreamSynchronize(s));
        for (int i = 0; i < n; i++) {
            const LbfgsState *sh = hs[i]->lb.st_host;
            st[i].iters[l] = sh->k;
            st[i].evals[l] = sh->evals;
            st[i].J[l] = sh->J;
            st[i].level_status[l] = sh->status == 1 ? REG_WARN_LINESEARCH : REG_OK;
            if (sh->status == -5 || sh->status == -6 || sh->status == -7)
                status = sh->status == -5 ? REG_ERR_NUMERIC : REG_ERR_TIMEOUT;
            else if (sh->status == 1 && status == REG_OK)
                status = REG_WARN_LINESEARCH;
            if (l == 0) {
                st[i].J_final = sh->J;
                st[i].D_final = sh->D;
                st[i].S_final = sh->S;
            }
        }
    }
    CK(cudaEventRecord(c0->lev_ev[0], s));
    for (int i = 0; i < n; i++)
        CK(cudaMemcpyAsync(u_out[i], hs[i]->lb.u, sizeof(float) * 3 * hs[i]->L[0].nn,
                           out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaFreeAsync(d.pl, s));
    CK(cudaFreeAsync(d.off, s));
    CK(cudaFreeAsync(d.counters, s));
    CK(cudaStreamSynchronize(s));
    double lsec[REG_MAX_LEVELS] = {};
    if (status >= 0)
        for (int l = start; l >= 0; l--) {   // level l ran from event l + 1 to event l
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c0->lev_ev[l + 1], c0->lev_ev[l]));
            lsec[l] = 1e-3 * ms;
        }
    for (int i = 0; i < n; i++) {
        for (int l = 0; l < REG_MAX_LEVELS; l++)
            st[i].level_seconds[l] = lsec[l];
        st[i].status = status;
        st[i].kernel_launches = launches;
        if (stats)
            stats[i] = st[i];
    }
    if (status < 0)
        return set_err(nullptr, status, "reg_register_batch: a pair ended with a numeric or loop-bound error");
    return status;
}
