// Fused objective pass for ratio-2 grids (every image dimension even and
// n_d = m_d / 2 + 1, the default rule): one kernel computes, per voxel,
//   y-hat = P u (Eq. 1), T(x + y-hat) and its interpolant gradient,
//   the NGF residual of Eq. 2 and v = d psi / d grad T,
//   g = adjoint central difference of v, r = g grad T (the chain rule),
// and reduces r to per-tile partial node sums of P^T r (Eq. 3).  From the node
// planes it holds anyway it also forms the curvature Laplacian w = mask L u of
// the nodes the tile owns and their share of S (Sec. 2.1).  A second,
// node-parallel kernel adds up the (at most 8) tile partials of each node and
// the curvature gradient alpha hbar_y L^T w.  Nothing per voxel goes to HBM.
//
// Tiling.  A CTA of 16 x 16 threads owns a 32 x 16 block of voxel columns:
// thread (tx, ty) holds the two adjacent columns 2 tx and 2 tx + 1 of row ty.
// The inner 28 x 12 columns are the output tile; the 2-voxel halo is what the
// stencil chain T~ -> a -> v -> g reaches.  The CTA marches along z through a
// segment of TZ output planes.  Two CTAs are resident per SM: each step ends
// in a block barrier, and while one CTA's warps wait there (or all stall in
// the same phase of the step) the other CTA's warps issue.  A 32 x 32 block
// of one 512-thread CTA per SM wastes less on the halo (1.31 against 1.52
// computed columns per output column) but ran 7 % slower.  With ratio 2 the P weights are 1/4 and 3/4;
// tiles start at even x, so the two columns of a thread always lie in the
// same node interval (x weights 1/4 and 3/4 of the same nodes), and the node
// loads, P's integer cell and the x reduction of P^T are shared by the pair.
// A node gathers voxels 2k-2 .. 2k+1 with weights 1/4, 3/4, 3/4, 1/4 per
// dimension, so an output tile of 28 x 12 x TZ voxels feeds 15 x 7 x
// (TZ/2 + 1) nodes; neighbouring tiles share one node plane per dimension and
// the gather kernel sums them.
//
// Arithmetic.  The two columns of a thread run the same computation, so every
// per-column quantity is a float2 pair (.x the first column, .y the second)
// and the FP32 work is issued as packed two-lane instructions (fma/add/mul/sub
// .f32x2): one issue slot serves both voxels.
//
// Template samples.  Handles keep a copy of T with a 2-voxel zero border on
// every side (PAD): a sample cell is clamped into the border with one unsigned
// min per axis, which reads the zero extension of R5 for any cell outside the
// image, and the 8 corners load without tests.  Callers that pass their own
// unpadded T (the allocation-free entry point) take bounds-tested loads.
//
// Scale factors.  The constant factors of r = (hbar / 2) g' (grad T') / h_c
// are left to the gather: the pass accumulates g' (the unscaled adjoint
// stencil of v) times the unscaled interpolant differences, and the gather
// multiplies component c by hbar / (2 h_c).
//
// Pipeline.  Step s works on plane zA = z0 - 2 + s and the lagging planes
//   A-finish zA    : interpolate T at both columns from the corners loaded
//                    last step
//   A-issue  zA+1  : at the first plane of a node interval, P on the interval
//                    (both planes) and the cp.async of the node-plane tile two
//                    intervals ahead; at its second plane, the trial node
//                    values u + t dir of the plane that copy brought; the
//                    coordinates of plane zA+1 and the loads of its 2 x 8
//                    corners and of R into registers, first used one step later
//   B  zA-2        : v from T~ and R planes zA-3 .. zA-1
//   C  zA-4        : r from v planes zA-5 .. zA-3; x reduction to node columns
//   D  zA-5        : y reduction of last step's rows, accumulation along z
// Every phase reads only what earlier steps wrote, so one barrier per step
// suffices, and the global loads of a plane overlap a whole step of compute.
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <queue>
#include <type_traits>
#include <vector>

#include "batch.h"
#include "internal.h"
#include "lbfgs_control.cuh"
#include "ngf_math.cuh"

#include "fused_pass.cuh"

namespace {

template <bool HAS_DIR, typename IMG = float, bool PAD = true, bool CURV = false>
__global__ void __launch_bounds__(BX * BY, CTAS_PER_SM) k_ngf_fused(FusedArgs a)
{
    extern __shared__ float sm[];
    fused_tile<HAS_DIR, IMG, PAD, CURV>(a, blockIdx.x, sm);
}

// Batched fused pass: a persistent grid walks the tiles of all pairs.  Mode 0
// evaluates at u; mode 1 at the trial point, for the pairs still searching.
template <bool HAS_DIR, typename IMG>
__global__ void __launch_bounds__(BX * BY, CTAS_PER_SM) k_ngf_fused_batch(const PairLevel *__restrict__ pl,
                                                                const int *__restrict__ tile_off, int npairs,
                                                                int total)
{
    extern __shared__ float sm[];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int p = find_pair(tile_off, npairs, item);
        const PairLevel &P = pl[p];
        if (HAS_DIR && !(P.st->active && P.st->ls_continue))
            continue;   // uniform over the CTA
        const FusedArgs &a = HAS_DIR ? P.fa_trial : P.fa_init;
        fused_tile<HAS_DIR, IMG, true, true>(a, item - __ldg(tile_off + p), sm);
        __syncthreads();   // the next tile reuses the shared rings
    }
}

__global__ void __launch_bounds__(GATHER_NODES) k_gather_grad(LevelGeom g, const float *__restrict__ part,
                                                              FusedSplit sp, int ntx, int nty,
                                                              const float *__restrict__ w, float alpha_hy,
                                                              float *__restrict__ grad)
{
    gather_grad_body(g, part, sp, ntx, nty, w, alpha_hy, grad, blockIdx.x, blockIdx.y);
}

// The end of an evaluation in the gather launch.  The final reduction reads
// only the D and S block partials of the kernels before, not the gradient, so
// block 0 reduces them into scal = [J, D, S] (the fixed order of
// finalize_body) and, for phase >= 0, takes that L-BFGS control phase (the
// Armijo decision of a trial point) first, while the other blocks gather.
struct FinArgs {
    const double *pD, *pS;  // block partials of D (fused tiles) and S (curvature blocks)
    int nD, nS;
    double hbar_half, alpha, hy_half;
    double *scal;
    int phase;              // -1: no control phase
    LbfgsState *st;
    unsigned long long h_ls;
};

__global__ void __launch_bounds__(GATHER_NODES) k_gather_fin(LevelGeom g, const float *__restrict__ part,
                                                             FusedSplit sp, int ntx, int nty,
                                                             const float *__restrict__ w, float alpha_hy,
                                                             float *__restrict__ grad, FinArgs f)
{
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        finalize_body(f.pD, f.nD, f.pS, f.nS, f.hbar_half, f.alpha, f.hy_half, f.scal);
        if (f.phase >= 0) {
            __syncthreads();
            lb_control_body(f.phase, f.st, nullptr, nullptr, 0, f.scal, f.h_ls, 0ULL, 0ULL);
        }
    }
    gather_grad_body(g, part, sp, ntx, nty, w, alpha_hy, grad, blockIdx.x, blockIdx.y);
}

}  // namespace

bool fused_eligible(const Level &L)
{
    for (int d = 0; d < 3; d++)
        if ((L.m[d] & 1) || L.n[d] != L.m[d] / 2 + 1)
            return false;
    return true;
}

// z segment lengths the throughput rule picks from (even: a segment covers
// whole node intervals)
constexpr int TZ_CAND[] = {2, 4, 8, 16, 32, 64, 128};

// Pipeline steps a segment pays beyond its planes (fill and drain)
constexpr int FUSED_FILL = 7;
// longest z segment cfg.fused_tz may force
constexpr int TZ_MAX = 512;

static int fused_cols(const int m[3]) { return ((m[0] + OX - 1) / OX) * ((m[1] + OY - 1) / OY); }

FusedSplit fused_split_uniform(int tz, int mz)
{
    FusedSplit sp;
    sp.l1 = tz;
    sp.n1 = mz / tz;
    sp.lr = mz - sp.n1 * tz;   // even, as mz and tz are
    return sp;
}

// Even z segment lengths that cut a depth of mz planes into ntz = 1, 2, ...
// nearly equal segments, tz = 2 ceil(mz / (2 ntz)), longest first, each once.
static std::vector<int> tz_splits(int mz)
{
    std::vector<int> v;
    for (int ntz = 1;; ntz++) {
        const int tz = 2 * ((mz + 2 * ntz - 1) / (2 * ntz));
        if (tz <= TZ_MAX && (v.empty() || tz < v.back()))
            v.push_back(tz);
        if (tz <= 2)
            break;
    }
    return v;
}

// Load model of the pass.  A tile costs its planes + 7 steps, times a weight
// for the share of its 32 x 16 columns inside the image (columns outside skip
// the loads, the interpolation and the NGF work; about a third of a step's
// work remains).  CTAS_PER_SM CTAs are resident per SM, each a slot, and the
// next free slot takes the next tile in launch order (tile_seg_col), so the
// model replays that order and returns the time the last slot finishes.
struct SplitModel {
    std::vector<double> colw;   // weight of each tile column, in column order
    int mz, sms;
    SplitModel(const int m[3], int num_sms) : mz(m[2]), sms(num_sms > 0 ? CTAS_PER_SM * num_sms : 1)
    {
        const int ntx = (m[0] + OX - 1) / OX, nty = (m[1] + OY - 1) / OY;
        auto frac = [](int t, int o, int width, int extent) {
            int n = 0;
            for (int i = t * o - 2; i < t * o - 2 + width; i++)
                n += i >= 0 && i < extent;
            return (double)n / width;
        };
        for (int ty = 0; ty < nty; ty++)
            for (int tx = 0; tx < ntx; tx++)
                colw.push_back(0.35 + 0.65 * frac(tx, OX, CW, m[0]) * frac(ty, OY, BY, m[1]));
    }
    double makespan(const FusedSplit &sp) const
    {
        // segment groups by length, longest first (stable), as tile_seg_col
        int len[3] = {sp.l1, sp.l2, sp.lr}, cnt[3] = {sp.n1, sp.n2, sp.lr > 0 ? 1 : 0};
        int ord[3] = {0, 1, 2};
        std::stable_sort(ord, ord + 3, [&](int x, int y) { return len[x] > len[y]; });
        std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
        for (int i = 0; i < sms; i++)
            free_at.push(0.0);
        double end = 0.0;
        for (int k = 0; k < 3; k++)
            for (int seg = 0; seg < cnt[ord[k]]; seg++)
                for (double w : colw) {
                    const double t = free_at.top() + w * (len[ord[k]] + FUSED_FILL);
                    free_at.pop();
                    free_at.push(t);
                    end = std::max(end, t);
                }
        return end;
    }
};

// Candidate splits of a depth: the equal splits, and for depths of 32 planes
// and more one or two segments of l1 planes, one to three of l2 < l1 and the
// remainder (lengths on a grid of mz / 32 planes).
static std::vector<FusedSplit> split_candidates(int mz)
{
    std::vector<FusedSplit> v;
    for (int tz : tz_splits(mz))
        v.push_back(fused_split_uniform(tz, mz));
    if (mz >= 32) {
        const int step = std::max(2, (mz / 32) & ~1);
        for (int l1 = step; l1 <= mz; l1 += step)
            for (int n1 = 1; n1 <= 2 && n1 * l1 <= mz; n1++)
                for (int l2 = step; l2 < l1; l2 += step)
                    for (int n2 = 1; n2 <= 3 && n1 * l1 + n2 * l2 <= mz; n2++) {
                        FusedSplit sp;
                        sp.l1 = l1;
                        sp.n1 = n1;
                        sp.l2 = l2;
                        sp.n2 = n2;
                        sp.lr = mz - n1 * l1 - n2 * l2;
                        v.push_back(sp);
                    }
    }
    return v;
}

// candidate splits, cheapest first under the load model (ties: fewer segments)
static std::vector<FusedSplit> splits_ranked(const int m[3], int num_sms)
{
    const SplitModel model(m, num_sms);
    std::vector<std::pair<double, FusedSplit>> r;
    for (const FusedSplit &sp : split_candidates(m[2]))
        r.push_back({model.makespan(sp), sp});
    std::stable_sort(r.begin(), r.end(), [](const std::pair<double, FusedSplit> &x,
                                            const std::pair<double, FusedSplit> &y) {
        if (x.first != y.first)
            return x.first < y.first;
        return x.second.count() < y.second.count();
    });
    std::vector<FusedSplit> v;
    for (auto &e : r)
        v.push_back(e.second);
    return v;
}

FusedSplit fused_split(const Level &L, int num_sms) { return L.split.valid() ? L.split : splits_ranked(L.m, num_sms)[0]; }

FusedSplit fused_split_plan(const int m[3], int num_sms, double *model_steps)
{
    const FusedSplit sp = splits_ranked(m, num_sms)[0];
    if (model_steps)
        *model_steps = SplitModel(m, num_sms).makespan(sp);
    return sp;
}

// Throughput rule: the z segment length of TZ_CAND with the fewest pipeline
// steps in total, ntz * (tz + 7) (ties: the longer one).  The right choice
// when other work keeps every SM busy (a batch of pairs); a single pair alone
// wants segments that fill the GPU in whole waves, which the load model and
// the autotuner find.
int fused_tz_throughput(const Level &L)
{
    int best = 0;
    long long best_steps = 0;
    for (int tz : TZ_CAND) {
        const long long steps = (long long)((L.m[2] + tz - 1) / tz) * (tz + FUSED_FILL);
        if (best == 0 || steps <= best_steps) {
            best = tz;
            best_steps = steps;
        }
    }
    return best;
}

bool fused_tz_valid(int tz) { return tz >= 2 && tz <= TZ_MAX && tz % 2 == 0; }

void fused_tile_shape(int *ox, int *oy, int *ctas_per_sm)
{
    *ox = OX;
    *oy = OY;
    *ctas_per_sm = CTAS_PER_SM;
}

// tile-partial floats of the level, for any split: a tile of a segment of len
// planes keeps len / 2 + 1 node planes, and the segments' lengths add up to
// the depth, so a split keeps at most depth / 2 + count <= depth planes per column
size_t fused_part_floats(const Level &L, int num_sms)
{
    (void)num_sms;
    return (size_t)fused_cols(L.m) * (size_t)(L.m[2] + 2) * NE;
}

FusedArgs fused_args(const reg_ctx *c, int level, const float *ub, const float *dir, const double *t_dev,
                     double *partials, int *ntiles)
{
    const Level &L = c->L[level];
    FusedArgs a;
    a.g = L.geom();
    const bool bf16 = c->cfg.image_dtype == 1 && L.Tb && L.Rb;
    a.T = bf16 ? static_cast<const void *>(L.Tb) : static_cast<const void *>(L.Tp);   // zero-bordered copies
    a.R = bf16 ? L.Rb : static_cast<const void *>(L.R);
    a.Rn = bf16 ? nullptr : L.Rn;
    a.ub = ub;
    a.dir = dir;
    a.t_dev = t_dev;
    a.tau = (float)c->cfg.tau;
    a.rho = (float)c->cfg.rho;
    a.split = fused_split(L, c->num_sms);
    a.ntx = (L.m[0] + OX - 1) / OX;
    a.nty = (L.m[1] + OY - 1) / OY;
    a.part = c->es.part;
    a.partials = partials;
    *ntiles = a.ntx * a.nty * a.split.count();
    a.w = c->es.w;
    a.partials_S = partials + *ntiles;   // the S partials follow the D partials
    return a;
}

cudaError_t launch_ngf_fused(reg_ctx *c, int level, const float *ub, const float *dir, const double *t_dev,
                             float *grad, double *partials, int *n_partials, cudaStream_t s)
{
    (void)grad;
    const Level &L = c->L[level];
    const bool bf16 = c->cfg.image_dtype == 1 && L.Tb && L.Rb;
    if (!bf16 && !L.Rn)
        return cudaErrorInvalidValue;   // FP32 handles keep R's normalized field beside the padded T
    int ntiles = 0;
    const FusedArgs a = fused_args(c, level, ub, dir, t_dev, partials, &ntiles);
    dim3 blk(BX, BY, 1), grd(ntiles, 1, 1);
    // the shared rings exceed the 48 KB default; the limit is set once per device
    static bool attr_set[64] = {};
    const int dev = c->device >= 0 && c->device < 64 ? c->device : 0;
    if (!attr_set[dev]) {
        cudaError_t e = set_fused_smem(k_ngf_fused<true, float>, smem_bytes<float, true, false>());
        if (e == cudaSuccess)
            e = set_fused_smem(k_ngf_fused<false, float>, smem_bytes<float, true, false>());
        if (e == cudaSuccess)
            e = set_fused_smem(k_ngf_fused<true, __nv_bfloat16>, smem_bytes<__nv_bfloat16, true, false>());
        if (e == cudaSuccess)
            e = set_fused_smem(k_ngf_fused<false, __nv_bfloat16>, smem_bytes<__nv_bfloat16, true, false>());
        if (e == cudaSuccess)
            e = set_fused_smem(k_ngf_fused<true, float, true, true>, smem_bytes<float, true, true>());
        if (e == cudaSuccess)
            e = set_fused_smem(k_ngf_fused<false, float, true, true>, smem_bytes<float, true, true>());
        if (e == cudaSuccess)
            e = set_fused_smem(k_ngf_fused<true, __nv_bfloat16, true, true>, smem_bytes<__nv_bfloat16, true, true>());
        if (e == cudaSuccess)
            e = set_fused_smem(k_ngf_fused<false, __nv_bfloat16, true, true>, smem_bytes<__nv_bfloat16, true, true>());
        if (e != cudaSuccess)
            return e;
        attr_set[dev] = true;
    }
    // the curvature Laplacian in the pass (the batched form's arithmetic) or beside it
    const bool curv = fused_curv_in_pass(c, level);
    if (bf16) {
        if (curv) {
            constexpr size_t SB = smem_bytes<__nv_bfloat16, true, true>();
            dir ? k_ngf_fused<true, __nv_bfloat16, true, true><<<grd, blk, SB, s>>>(a)
                : k_ngf_fused<false, __nv_bfloat16, true, true><<<grd, blk, SB, s>>>(a);
        } else {
            constexpr size_t SB = smem_bytes<__nv_bfloat16, true, false>();
            dir ? k_ngf_fused<true, __nv_bfloat16><<<grd, blk, SB, s>>>(a)
                : k_ngf_fused<false, __nv_bfloat16><<<grd, blk, SB, s>>>(a);
        }
    } else {
        if (curv) {
            constexpr size_t SB = smem_bytes<float, true, true>();
            dir ? k_ngf_fused<true, float, true, true><<<grd, blk, SB, s>>>(a)
                : k_ngf_fused<false, float, true, true><<<grd, blk, SB, s>>>(a);
        } else {
            constexpr size_t SB = smem_bytes<float, true, false>();
            dir ? k_ngf_fused<true, float><<<grd, blk, SB, s>>>(a)
                : k_ngf_fused<false, float><<<grd, blk, SB, s>>>(a);
        }
    }
    *n_partials = ntiles;
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_gather_fin(reg_ctx *c, int level, const float *w, float alpha_hy, float *grad, int nD,
                              const double *pS, int nS, double *scal, int phase, cudaStream_t s)
{
    const Level &L = c->L[level];
    const FusedSplit sp = fused_split(L, c->num_sms);
    const int ntx = (L.m[0] + OX - 1) / OX, nty = (L.m[1] + OY - 1) / OY;
    const dim3 gn = gather_grid(L.n);
    FinArgs f;
    f.pD = c->es.partials;
    f.nD = nD;
    f.pS = pS;
    f.nS = nS;
    f.hbar_half = 0.5 * L.h[0] * L.h[1] * L.h[2];
    f.alpha = c->cfg.alpha;
    f.hy_half = 0.5 * L.H[0] * L.H[1] * L.H[2];
    f.scal = scal;
    f.phase = phase;
    f.st = c->lb.st;
    f.h_ls = phase >= 0 ? lbfgs_graph_handle_ls() : 0ULL;
    k_gather_fin<<<gn, GATHER_NODES, 0, s>>>(L.geom(), c->es.part, sp, ntx, nty, w, alpha_hy, grad, f);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_gather_grad(reg_ctx *c, int level, const float *w, float alpha_hy, float *grad, cudaStream_t s)
{
    const Level &L = c->L[level];
    const FusedSplit sp = fused_split(L, c->num_sms);
    const int ntx = (L.m[0] + OX - 1) / OX, nty = (L.m[1] + OY - 1) / OY;
    k_gather_grad<<<gather_grid(L.n), GATHER_NODES, 0, s>>>(L.geom(), c->es.part, sp, ntx, nty, w, alpha_hy, grad);
    c->launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Autotuner of the z segmentation of the fused pass.  The candidates are the
// TUNE_CAND splits the load model ranks cheapest plus its two best equal
// splits (in case the model misjudges the weights); for each the pass runs on
// the level's own images at u = u_zero (one warm launch, then the median of
// three CUDA-event timings) and the fastest wins.  Short segments start more
// CTAs (small levels fill the GPU) but pay the 7 pipeline-fill steps and the
// shared node planes more often, and the last CTAs may leave SMs idle, so the
// best split depends on the level and the GPU.  Choices are cached per (image
// dims, SM count, image type, device) for the life of the process: handles of
// the same geometry tune once and pick the same tiling.
// ---------------------------------------------------------------------------
namespace {
constexpr int TUNE_CAND = 6;
std::mutex g_tune_mu;
std::map<std::array<int, 6>, FusedSplit> g_tune;
}

cudaError_t fused_autotune(reg_ctx *c, int level, const float *u_zero, cudaStream_t s)
{
    Level &L = c->L[level];
    const bool bf16 = c->cfg.image_dtype == 1 && L.Tb && L.Rb;
    const std::array<int, 6> key{L.m[0], L.m[1], L.m[2], c->num_sms, bf16 ? 1 : 0, c->device};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            L.split = it->second;
            return cudaSuccess;
        }
    }
    const std::vector<FusedSplit> ranked = splits_ranked(L.m, c->num_sms);
    std::vector<FusedSplit> cand;
    for (const FusedSplit &sp : ranked)
        if ((int)cand.size() < TUNE_CAND)
            cand.push_back(sp);
    int uniform = 0;
    for (const FusedSplit &sp : ranked) {
        if (uniform == 2)
            break;
        if (sp.n2 == 0 && (sp.lr == 0 || sp.n1 == 0)) {   // equal segments (no remainder)
            uniform++;
            if (std::find(cand.begin(), cand.end(), sp) == cand.end())
                cand.push_back(sp);
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    FusedSplit best;
    float best_ms = 0.f;
    for (const FusedSplit &sp : cand) {
        if (e != cudaSuccess)
            break;
        L.split = sp;
        int nD = 0;
        float t[3];
        for (int r = -1; r < 3 && e == cudaSuccess; r++) {   // r = -1: warm launch
            if (r >= 0)
                e = cudaEventRecord(e0, s);
            if (e == cudaSuccess)
                e = launch_ngf_fused(c, level, u_zero, nullptr, nullptr, nullptr, c->es.partials, &nD, s);
            if (e == cudaSuccess && r >= 0)
                e = cudaEventRecord(e1, s);
            if (e == cudaSuccess && r >= 0)
                e = cudaEventSynchronize(e1);
            if (e == cudaSuccess && r >= 0)
                e = cudaEventElapsedTime(&t[r], e0, e1);
        }
        if (e != cudaSuccess)
            break;
        const float med = fmaxf(fminf(t[0], t[1]), fminf(fmaxf(t[0], t[1]), t[2]));
        if (!best.valid() || med < best_ms) {
            best = sp;
            best_ms = med;
        }
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        L.split = FusedSplit();
        return e;
    }
    L.split = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Explicit-buffer launches of the fused pass and its gather, for callers that
// own every buffer themselves (the allocation-free entry point).  Geometry
// comes in as a LevelGeom of a ratio-2 grid; no per-dimension tables are used.
// The split is the load model's first choice for the dims (cached per dims).
// ---------------------------------------------------------------------------
static FusedSplit fused_split_dims(const int m[3], int num_sms)
{
    static std::mutex mu;
    static std::map<std::array<int, 4>, FusedSplit> cache;
    const std::array<int, 4> key{m[0], m[1], m[2], num_sms};
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end())
        return it->second;
    const FusedSplit sp = splits_ranked(m, num_sms)[0];
    cache[key] = sp;
    return sp;
}

void fused_layout_dims(const int m[3], int num_sms, int *tz, int *tiles, size_t *part_floats)
{
    const FusedSplit sp = fused_split_dims(m, num_sms);
    const int ncols = fused_cols(m);
    *tz = sp.longest();
    *tiles = ncols * sp.count();
    *part_floats = (size_t)ncols * sp.planes_before(sp.count()) * NE;
}

// the explicit-buffer pass reads the caller's unpadded T (bounds-tested corner loads)
cudaError_t fused_set_smem_limit()
{
    return set_fused_smem(k_ngf_fused<false, float, false, true>, smem_bytes<float, false, true>());
}

cudaError_t launch_ngf_fused_raw(const LevelGeom &g, const float *T, const float *R, const float *u, float tau,
                                 float rho, int num_sms, float *part, double *partials, float *w, cudaStream_t s)
{
    FusedArgs a;
    a.g = g;
    a.T = T;
    a.R = R;
    a.Rn = nullptr;
    a.ub = u;
    a.dir = nullptr;
    a.t_dev = nullptr;
    a.tau = tau;
    a.rho = rho;
    a.split = fused_split_dims(g.m, num_sms);
    a.ntx = (g.m[0] + OX - 1) / OX;
    a.nty = (g.m[1] + OY - 1) / OY;
    a.part = part;
    a.partials = partials;
    dim3 blk(BX, BY, 1), grd(a.ntx * a.nty * a.split.count(), 1, 1);
    a.w = w;
    a.partials_S = partials + grd.x;   // the S partials follow the D partials
    k_ngf_fused<false, float, false, true><<<grd, blk, smem_bytes<float, false, true>(), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gather_grad_raw(const LevelGeom &g, const float *part, int num_sms, const float *w,
                                   float alpha_hy, float *grad, cudaStream_t s)
{
    const FusedSplit sp = fused_split_dims(g.m, num_sms);
    const int ntx = (g.m[0] + OX - 1) / OX, nty = (g.m[1] + OY - 1) / OY;
    k_gather_grad<<<gather_grid(g.n), GATHER_NODES, 0, s>>>(g, part, sp, ntx, nty, w, alpha_hy, grad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched fused pass and gather over all pairs of a level (batch.cu)
// ---------------------------------------------------------------------------
static bool g_batch_attr_set[64] = {};

cudaError_t launch_fused_batch(const PairLevel *pl, const int *tile_off, int npairs, int total, int mode, bool bf16,
                               int grid, int device, cudaStream_t s)
{
    const int dev = device >= 0 && device < 64 ? device : 0;
    if (!g_batch_attr_set[dev]) {
        constexpr size_t BF = smem_bytes<float, true, true>(), BH = smem_bytes<__nv_bfloat16, true, true>();
        cudaError_t e = set_fused_smem(k_ngf_fused_batch<true, float>, BF);
        if (e == cudaSuccess)
            e = set_fused_smem(k_ngf_fused_batch<false, float>, BF);
        if (e == cudaSuccess)
            e = set_fused_smem(k_ngf_fused_batch<true, __nv_bfloat16>, BH);
        if (e == cudaSuccess)
            e = set_fused_smem(k_ngf_fused_batch<false, __nv_bfloat16>, BH);
        if (e != cudaSuccess)
            return e;
        g_batch_attr_set[dev] = true;
    }
    dim3 blk(BX, BY, 1);
    if (bf16) {
        constexpr size_t SB = smem_bytes<__nv_bfloat16, true, true>();
        if (mode)
            k_ngf_fused_batch<true, __nv_bfloat16><<<grid, blk, SB, s>>>(pl, tile_off, npairs, total);
        else
            k_ngf_fused_batch<false, __nv_bfloat16><<<grid, blk, SB, s>>>(pl, tile_off, npairs, total);
    } else {
        constexpr size_t SB = smem_bytes<float, true, true>();
        if (mode)
            k_ngf_fused_batch<true, float><<<grid, blk, SB, s>>>(pl, tile_off, npairs, total);
        else
            k_ngf_fused_batch<false, float><<<grid, blk, SB, s>>>(pl, tile_off, npairs, total);
    }
    return cudaGetLastError();
}

namespace {

__global__ void __launch_bounds__(GATHER_NODES) k_gather_batch(const PairLevel *__restrict__ pl, const int *__restrict__ off,
                                                      int npairs, int total, int mode)
{
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int p = find_pair(off, npairs, item);
        const PairLevel &P = pl[p];
        if (mode == 1 && !(P.st->active && P.st->ls_continue))
            continue;
        const int lin = item - __ldg(off + p);
        const FusedArgs &a = P.fa_init;
        gather_grad_body(P.geom, a.part, a.split, a.ntx, a.nty, P.w, P.alpha_hy, mode ? P.gt : P.g, lin % P.gbx,
                         lin / P.gbx);
    }
}

}  // namespace

cudaError_t launch_gather_batch(const PairLevel *pl, const int *off, int npairs, int total, int mode, int grid,
                                cudaStream_t s)
{
    k_gather_batch<<<grid, GATHER_NODES, 0, s>>>(pl, off, npairs, total, mode);
    return cudaGetLastError();
}

// tiling of a level of the fused pass, for the batch descriptors
void fused_tiling(const Level &L, int num_sms, FusedSplit *split, int *ntx, int *nty)
{
    *split = fused_split(L, num_sms);
    *ntx = (L.m[0] + OX - 1) / OX;
    *nty = (L.m[1] + OY - 1) / OY;
}
