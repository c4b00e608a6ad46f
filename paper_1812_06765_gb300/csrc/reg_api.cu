// C ABI of libreg.so (declared in include/reg.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "internal.h"

namespace {

thread_local std::string g_create_err;

void free_level(Level &L)
{
    cudaFree(L.R);
    cudaFree(L.T);
    cudaFree(L.Tp);
    cudaFree(L.Rn);
    cudaFree(L.Rb);
    cudaFree(L.Tb);
    for (int d = 0; d < 3; d++) {
        cudaFree(L.pk0[d]);
        cudaFree(L.pw1[d]);
        cudaFree(L.tfirst[d]);
        cudaFree(L.tcnt[d]);
        cudaFree(L.tw[d]);
        cudaFree(L.qk0[d]);
        cudaFree(L.qw1[d]);
    }
    L = Level();
}

void free_buffers(reg_ctx *c)
{
    for (int l = 0; l < REG_MAX_LEVELS; l++) {
        free_level(c->L[l]);
        if (c->iter_graph[l]) cudaGraphExecDestroy(c->iter_graph[l]);
        if (c->init_graph[l]) cudaGraphExecDestroy(c->init_graph[l]);
        c->iter_graph[l] = nullptr;
        c->init_graph[l] = nullptr;
    }
    EvalScratch &e = c->es;
    cudaFree(e.Tw);
    cudaFree(e.dT);
    cudaFree(e.v);
    cudaFree(e.r);
    cudaFree(e.w);
    cudaFree(e.part);
    cudaFree(e.partials);
    cudaFree(e.scal);
    c->es = EvalScratch();
    LbfgsBuffers &b = c->lb;
    cudaFree(b.u);
    cudaFree(b.pdir);
    cudaFree(b.g);
    cudaFree(b.gt);
    cudaFree(b.P);
    cudaFree(b.Y);
    cudaFree(b.partials);
    cudaFree(b.gpart);
    cudaFree(b.gbar);
    cudaFree(b.cnt);
    cudaFree(b.st);
    cudaFree(b.scal_t);
    if (b.st_host) cudaFreeHost(b.st_host);
    c->lb = LbfgsBuffers();
    c->have_images = false;
}

// cfg.fused_split: all zero, or counts >= 0 and even lengths in 2 .. 512 for
// every group that is used, at least one segment
static bool split_config_valid(const int v[5])
{
    if (!v[0] && !v[1] && !v[2] && !v[3] && !v[4])
        return true;
    if (v[1] < 0 || v[3] < 0 || v[0] < 0 || v[2] < 0 || v[4] < 0)
        return false;
    auto len_ok = [](int l) { return l >= 2 && l <= 512 && l % 2 == 0; };
    if ((v[1] > 0 && !len_ok(v[0])) || (v[3] > 0 && !len_ok(v[2])) || (v[4] > 0 && !len_ok(v[4])))
        return false;
    return v[1] + v[3] + (v[4] > 0 ? 1 : 0) > 0;
}

static FusedSplit split_from_config(const int v[5])
{
    FusedSplit sp;
    sp.l1 = v[0];
    sp.n1 = v[1];
    sp.l2 = v[2];
    sp.n2 = v[3];
    sp.lr = v[4];
    return sp;
}

int validate_config(const reg_config *cfg, std::string &msg)
{
    char buf[256];
    if (!(cfg->tau > 0) || !(cfg->rho > 0)) msg = "tau and rho must be > 0";
    else if (!(cfg->alpha >= 0)) msg = "alpha must be >= 0";
    else if (!(cfg->c1 > 0 && cfg->c1 < 1)) msg = "c1 must be in (0, 1)";
    else if (cfg->levels < 1 || cfg->levels > REG_MAX_LEVELS) {
        snprintf(buf, sizeof buf, "levels must be in 1..%d", REG_MAX_LEVELS);
        msg = buf;
    } else if (cfg->lbfgs_mem < 1 || cfg->lbfgs_mem > REG_MAX_MEM) {
        snprintf(buf, sizeof buf, "lbfgs_mem must be in 1..%d", REG_MAX_MEM);
        msg = buf;
    } else if (cfg->max_backtracks < 1) msg = "max_backtracks must be >= 1";
    else if (cfg->start_level >= cfg->levels) msg = "start_level must be < levels";
    else if (cfg->eval_impl < 0 || cfg->eval_impl > 3) msg = "eval_impl must be 0, 1, 2 or 3";
    else if (cfg->image_dtype != 0 && cfg->image_dtype != 1) msg = "image_dtype must be 0 (FP32) or 1 (BF16)";
    else if (!(cfg->tol_grad_rel >= 0) || !(cfg->tol_j_rel >= 0)) msg = "tolerances must be >= 0";
    else if (cfg->autotune != 0 && cfg->autotune != 1) msg = "autotune must be 0 or 1";
    else if (cfg->test_expire_wait != 0 && cfg->test_expire_wait != 1) msg = "test_expire_wait must be 0 or 1";
    else if (!split_config_valid(cfg->fused_split))
        msg = "fused_split must be all 0 or (l1, n1, l2, n2, lr): counts >= 0, lengths even, 2 .. 512 where used";
    else if (cfg->fused_tz != 0 && cfg->fused_tz != -1 && !fused_tz_valid(cfg->fused_tz))
        msg = "fused_tz must be 0, -1 or an even length in 2 .. 512";
    else return REG_OK;
    return REG_ERR_ARG;
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src)
{
    cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * (src.empty() ? 1 : src.size()));
    if (e != cudaSuccess) return e;
    if (src.empty()) return cudaSuccess;
    return cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

// Per-dimension tables of P (voxel i -> node k0, weight of k0 + 1) and of P^T
// (node k -> first voxel, count, weights), from the hat functions at voxel
// centres t = (i + 1/2) h / H (Sec. 2.2, Eq. 3: weights and index sets are
// determined beforehand, separately for each dimension).  Host only.
struct AxisTables {
    std::vector<int> k0, first, cnt;
    std::vector<float> w1, tw;   // tw[k * maxw + j]: weight of voxel first[k] + j for node k
    int maxw = 1;
};

AxisTables axis_tables(int m, double h, double H, int n)
{
    AxisTables a;
    a.k0.resize(m);
    a.w1.resize(m);
    std::vector<double> t(m);
    for (int i = 0; i < m; i++) {
        t[i] = (i + 0.5) * h / H;
        int k = (int)floor(t[i]);
        if (k > n - 2) k = n - 2;
        if (k < 0) k = 0;
        a.k0[i] = k;
        a.w1[i] = (float)(t[i] - k);
    }
    a.first.assign(n, 0);
    a.cnt.assign(n, 0);
    std::vector<std::vector<double>> ws(n);
    for (int k = 0; k < n; k++) {
        for (int i = 0; i < m; i++) {
            double w = 1.0 - fabs(t[i] - k);
            if (w > 0.0) {
                if (ws[k].empty()) a.first[k] = i;
                ws[k].push_back(w);
            }
        }
        a.cnt[k] = (int)ws[k].size();
        if (a.cnt[k] > a.maxw) a.maxw = a.cnt[k];
    }
    a.tw.assign((size_t)n * a.maxw, 0.f);
    for (int k = 0; k < n; k++)
        for (int j = 0; j < a.cnt[k]; j++) a.tw[(size_t)k * a.maxw + j] = (float)ws[k][j];
    return a;
}

cudaError_t build_tables(Level &L)
{
    for (int d = 0; d < 3; d++) {
        const AxisTables a = axis_tables(L.m[d], L.h[d], L.H[d], L.n[d]);
        L.tmaxw[d] = a.maxw;
        cudaError_t e;
        if ((e = upload(&L.pk0[d], a.k0)) != cudaSuccess) return e;
        if ((e = upload(&L.pw1[d], a.w1)) != cudaSuccess) return e;
        if ((e = upload(&L.tfirst[d], a.first)) != cudaSuccess) return e;
        if ((e = upload(&L.tcnt[d], a.cnt)) != cudaSuccess) return e;
        if ((e = upload(&L.tw[d], a.tw)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Prolongation tables of a fine level from the next coarser one: fine node j
// at j H_f in mm, coarse coordinate j H_f / H_c.
cudaError_t build_prolong_tables(Level &F, const Level &C)
{
    for (int d = 0; d < 3; d++) {
        std::vector<int> k0(F.n[d]);
        std::vector<float> w1(F.n[d]);
        for (int j = 0; j < F.n[d]; j++) {
            double t = j * F.H[d] / C.H[d];
            if (t > C.n[d] - 1) t = C.n[d] - 1;
            int k = (int)floor(t);
            if (k > C.n[d] - 2) k = C.n[d] - 2;
            k0[j] = k;
            w1[j] = (float)(t - k);
        }
        cudaError_t e;
        if ((e = upload(&F.qk0[d], k0)) != cudaSuccess) return e;
        if ((e = upload(&F.qw1[d], w1)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

LevelGeom Level::geom() const
{
    LevelGeom g;
    for (int d = 0; d < 3; d++) {
        g.m[d] = m[d];
        g.n[d] = n[d];
        g.h[d] = (float)h[d];
        g.ih[d] = (float)(1.0 / h[d]);
        g.iH2[d] = (float)(1.0 / (H[d] * H[d]));
        g.pk0[d] = pk0[d];
        g.pw1[d] = pw1[d];
        g.tfirst[d] = tfirst[d];
        g.tcnt[d] = tcnt[d];
        g.tw[d] = tw[d];
        g.tmaxw[d] = tmaxw[d];
    }
    g.hbar = (float)(h[0] * h[1] * h[2]);
    g.hbar_y = (float)(H[0] * H[1] * H[2]);
    g.nv = nv;
    g.nn = nn;
    return g;
}

int set_err(reg_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_err = buf;
    return code;
}

int cuda_err(reg_ctx *c, cudaError_t e, const char *what)
{
    return set_err(c, e == cudaErrorMemoryAllocation ? REG_ERR_OOM : REG_ERR_CUDA, "%s: %s (%s)", what,
                   cudaGetErrorString(e), cudaGetErrorName(e));
}

// Device buffers of a new image geometry: level images and tables, evaluation
// scratch and the L-BFGS vectors (all sized by the finest level).
int allocate_buffers(reg_ctx *c)
{
    const reg_config &cfg = c->cfg;
    long long nmax = 0;
    int maxpart = 0;
    for (int l = 0; l < c->levels; l++) {
        Level &L = c->L[l];
        CK(cudaMalloc(&L.R, sizeof(float) * L.nv));
        CK(cudaMalloc(&L.T, sizeof(float) * L.nv));
        CK(build_tables(L));
        if (l > 0) CK(build_prolong_tables(c->L[l - 1], L));
        if (3 * L.nn > nmax) nmax = 3 * L.nn;
        int p = eval_partials_needed(L);
        if (p > maxpart) maxpart = p;
    }
    EvalScratch &es = c->es;
    long long mp_vox = 0;      // largest level served by the multi-pass kernels
    size_t part = 0;           // largest tile-partial buffer of the fused pass
    for (int l = 0; l < c->levels; l++) {
        if (use_fused(c, l)) {
            size_t p = fused_part_floats(c->L[l], c->num_sms);
            if (p > part) part = p;
        } else if (c->L[l].nv > mp_vox) {
            mp_vox = c->L[l].nv;
        }
    }
    if (mp_vox > 0) {
        CK(cudaMalloc(&es.Tw, sizeof(float) * mp_vox));
        CK(cudaMalloc(&es.dT, sizeof(float) * 3 * mp_vox));
        CK(cudaMalloc(&es.v, sizeof(float) * 3 * mp_vox));
        CK(cudaMalloc(&es.r, sizeof(float) * 3 * mp_vox));
    }
    if (part > 0) {
        CK(cudaMalloc(&es.part, sizeof(float) * part));
        es.part_floats = part;
    }
    // the fused pass reads T through a zero-bordered copy (FP32, or BF16 beside a BF16 R)
    for (int l = 0; l < c->levels; l++)
        if (use_fused(c, l)) {
            const long long np = padded_voxels(c->L[l].m);
            if (cfg.image_dtype == 1) {
                CK(cudaMalloc(&c->L[l].Rb, sizeof(__nv_bfloat16) * c->L[l].nv));
                CK(cudaMalloc(&c->L[l].Tb, sizeof(__nv_bfloat16) * np));
            } else {
                CK(cudaMalloc(&c->L[l].Tp, sizeof(float) * np));
                CK(cudaMalloc(&c->L[l].Rn, sizeof(float4) * c->L[l].nv));
            }
        }
    CK(cudaMalloc(&es.w, sizeof(float) * nmax));
    CK(cudaMalloc(&es.partials, sizeof(double) * maxpart));
    CK(cudaMalloc(&es.scal, sizeof(double) * 4));
    es.max_partials = maxpart;
    LbfgsBuffers &b = c->lb;
    b.n = nmax;
    b.slots = cfg.lbfgs_mem + 1;
    CK(cudaMalloc(&b.u, sizeof(float) * nmax));
    CK(cudaMalloc(&b.pdir, sizeof(float) * nmax));
    CK(cudaMalloc(&b.g, sizeof(float) * nmax));
    CK(cudaMalloc(&b.gt, sizeof(float) * nmax));
    const long long nring = (nmax + 3) & ~3LL;   // slot stride rounded up to 16 bytes
    CK(cudaMalloc(&b.P, sizeof(float) * nring * b.slots));
    CK(cudaMalloc(&b.Y, sizeof(float) * nring * b.slots));
    // the largest per-block layout is that of reg_lbfgs_direction's pair dots
    b.max_partials = 4 * c->num_sms * (2 + 2 * LB_MAXM + 2 * LB_MAXM * LB_MAXM) + 1024;
    CK(cudaMalloc(&b.partials, sizeof(float) * b.max_partials));
    {   // group sums and arrival counters of the vector passes (<= 4 blocks per SM)
        const int groups = (4 * c->num_sms + LB_RG - 1) / LB_RG;
        CK(cudaMalloc(&b.gpart, sizeof(float2) * groups * (2 + 4 * LB_MAXS)));
        b.cnt_len = groups + 1;
        CK(cudaMalloc(&b.cnt, sizeof(unsigned) * b.cnt_len));
        CK(cudaMemset(b.cnt, 0, sizeof(unsigned) * b.cnt_len));
        CK(cudaMalloc(&b.gbar, 3 * sizeof(unsigned)));
        CK(cudaMemset(b.gbar, 0, 3 * sizeof(unsigned)));
    }
    CK(cudaMalloc(&b.st, sizeof(LbfgsState)));
    CK(cudaMalloc(&b.scal_t, sizeof(double) * 4));
    CK(cudaMallocHost(&b.st_host, sizeof(LbfgsState)));
    CK(cudaMemsetAsync(b.st, 0, sizeof(LbfgsState), c->stream));
    return REG_OK;
}

extern "C" {

int reg_version(void) { return 10000; }

void reg_config_default(reg_config *cfg)
{
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->tau = cfg->rho = 0.01;
    cfg->alpha = 10.0;
    cfg->c1 = 1e-4;
    cfg->tol_grad_rel = 1e-5;
    cfg->tol_j_rel = 1e-7;
    cfg->tol_j_count = 3;
    cfg->levels = 1;
    cfg->lbfgs_mem = 5;
    cfg->max_backtracks = 20;
    cfg->fixed_iters = 0;
    cfg->start_level = -1;
    for (int l = 0; l < REG_MAX_LEVELS; l++) cfg->max_iter[l] = 50;
    cfg->eval_impl = 0;
    cfg->use_graph = 1;
    cfg->autotune = 1;
    cfg->fused_tz = 0;
}

int reg_create(reg_handle *out, const reg_config *cfg, void *cuda_stream)
{
    if (!out || !cfg) return set_err(nullptr, REG_ERR_ARG, "reg_create: NULL argument");
    *out = nullptr;
    std::string msg;
    if (validate_config(cfg, msg) != REG_OK) return set_err(nullptr, REG_ERR_ARG, "reg_create: %s", msg.c_str());
    reg_ctx *c = new reg_ctx();
    c->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = lbfgs_kernels_setup(c->device);
    if (e == cudaSuccess) {
        // NULL is the legacy default stream (ordered with every blocking stream)
        c->stream = (cudaStream_t)cuda_stream;
        c->own_stream = false;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_side, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&c->kev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&c->kev[1]);
    if (e != cudaSuccess) {
        set_err(nullptr, REG_ERR_CUDA, "reg_create: %s", cudaGetErrorString(e));
        reg_destroy(c);
        return REG_ERR_CUDA;
    }
    *out = c;
    return REG_OK;
}

int reg_set_images(reg_handle c, const float *R, const float *T, const int dims[3], const double spacing_mm[3],
                   int ptr_is_device)
{
    if (!c) return set_err(nullptr, REG_ERR_ARG, "reg_set_images: NULL handle");
    if (!R || !T || !dims || !spacing_mm) return set_err(c, REG_ERR_ARG, "reg_set_images: NULL argument");
    for (int d = 0; d < 3; d++) {
        if (dims[d] < 4) return set_err(c, REG_ERR_ARG, "reg_set_images: dims[%d] = %d < 4", d, dims[d]);
        if (!(spacing_mm[d] > 0) || !isfinite(spacing_mm[d]))
            return set_err(c, REG_ERR_ARG, "reg_set_images: spacing[%d] must be finite and > 0", d);
    }
    // the kernels index a volume with 32-bit integers and launch one grid row per plane
    if ((long long)dims[0] * dims[1] * dims[2] > REG_MAX_VOXELS || dims[2] > REG_MAX_PLANES)
        return set_err(c, REG_ERR_ARG, "reg_set_images: %d x %d x %d voxels (at most %lld voxels and %d planes)",
                       dims[0], dims[1], dims[2], (long long)REG_MAX_VOXELS, REG_MAX_PLANES);
    CK(cudaStreamSynchronize(c->stream));
    const reg_config &cfg = c->cfg;
    // geometry of every level
    Level G[REG_MAX_LEVELS];
    for (int l = 0; l < cfg.levels; l++) {
        Level &L = G[l];
        for (int d = 0; d < 3; d++) {
            L.m[d] = l == 0 ? dims[d] : (G[l - 1].m[d] + 1) / 2;
            L.h[d] = l == 0 ? spacing_mm[d] : 2.0 * G[l - 1].h[d];
            L.n[d] = cfg.node_dims[l][d] > 0 ? cfg.node_dims[l][d] : L.m[d] / 2 + 1;
            if (L.m[d] < 4 || L.n[d] < 3)
                return set_err(c, REG_ERR_ARG,
                               "reg_set_images: level %d has %d voxels / %d nodes in dim %d (need >= 4 / >= 3)",
                               l, L.m[d], L.n[d], d);
            L.H[d] = L.m[d] * L.h[d] / (L.n[d] - 1);
        }
        L.nv = (long long)L.m[0] * L.m[1] * L.m[2];
        L.nn = (long long)L.n[0] * L.n[1] * L.n[2];
        if (3 * L.nn > REG_MAX_VOXELS || L.n[2] > REG_MAX_PLANES)
            return set_err(c, REG_ERR_ARG,
                           "reg_set_images: level %d has %d x %d x %d nodes (at most %lld unknowns and %d node planes)",
                           l, L.n[0], L.n[1], L.n[2], (long long)REG_MAX_VOXELS, REG_MAX_PLANES);
    }
    // the same grid sizes again: keep every buffer and table (the tables depend
    // only on voxel and node counts), update the spacings
    bool reuse = c->have_images && c->levels == cfg.levels;
    for (int l = 0; reuse && l < cfg.levels; l++)
        for (int d = 0; d < 3; d++)
            reuse = reuse && c->L[l].m[d] == G[l].m[d] && c->L[l].n[d] == G[l].n[d];
    if (reuse) {
        bool same_spacing = true;
        for (int l = 0; l < cfg.levels; l++)
            for (int d = 0; d < 3; d++)
                same_spacing = same_spacing && c->L[l].h[d] == G[l].h[d];
        if (!same_spacing)   // graphs bake the spacings into their kernel arguments
            for (int l = 0; l < REG_MAX_LEVELS; l++)
                if (c->iter_graph[l]) {
                    cudaGraphExecDestroy(c->iter_graph[l]);
                    c->iter_graph[l] = nullptr;
                }
        for (int l = 0; l < cfg.levels; l++)
            for (int d = 0; d < 3; d++) {
                c->L[l].h[d] = G[l].h[d];
                c->L[l].H[d] = G[l].H[d];
            }
    } else {
        free_buffers(c);
        c->levels = cfg.levels;
        for (int l = 0; l < c->levels; l++) {
            Level &L = c->L[l];
            for (int d = 0; d < 3; d++) {
                L.m[d] = G[l].m[d];
                L.n[d] = G[l].n[d];
                L.h[d] = G[l].h[d];
                L.H[d] = G[l].H[d];
            }
            L.nv = G[l].nv;
            L.nn = G[l].nn;
        }
        int r = allocate_buffers(c);
        if (r != REG_OK) return r;
    }
    const long long nv0 = c->L[0].nv;
    c->have_images = false;

    // finest images, then the pyramid: R on the handle's stream, T on the side stream
    cudaMemcpyKind kind = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaEventRecord(c->ev_side, c->stream));
    CK(cudaStreamWaitEvent(c->side, c->ev_side, 0));
    CK(cudaMemcpyAsync(c->L[0].R, R, sizeof(float) * nv0, kind, c->stream));
    CK(cudaMemcpyAsync(c->L[0].T, T, sizeof(float) * nv0, kind, c->side));
    for (int l = 1; l < c->levels; l++) {
        CK(launch_restrict(c->L[l - 1].R, c->L[l - 1].m, c->L[l].R, c->stream));
        CK(launch_restrict(c->L[l - 1].T, c->L[l - 1].m, c->L[l].T, c->side));
        c->launches += 2;
    }
    CK(cudaEventRecord(c->ev_side, c->side));
    CK(cudaStreamWaitEvent(c->stream, c->ev_side, 0));
    for (int l = 0; l < c->levels; l++) {   // the fused pass's copies; BF16 rounded to nearest even
        if (c->L[l].Rb) {
            CK(launch_to_bf16(c->L[l].R, c->L[l].Rb, c->L[l].nv, c->stream));
            CK(launch_pad_template(c->L[l].T, c->L[l].m, c->L[l].Tb, c->stream));
            c->launches += 2;
        }
        if (c->L[l].Tp) {
            CK(launch_pad_template(c->L[l].T, c->L[l].m, c->L[l].Tp, c->stream));
            CK(launch_ref_normal_field(c->L[l], cfg.rho, c->stream));
            c->launches += 2;
        }
    }
    // tiling of the fused pass per level: forced, autotuned (at u = 0, with the
    // direction buffer as the zero field) or the default rule
    for (int l = 0; l < c->levels; l++) {
        if (!use_fused(c, l) || c->L[l].split.valid())
            continue;
        const FusedSplit forced = split_from_config(cfg.fused_split);
        if (forced.valid() && forced.n1 * forced.l1 + forced.n2 * forced.l2 + forced.lr == c->L[l].m[2]) {
            c->L[l].split = forced;
        } else if (cfg.fused_tz > 0) {
            c->L[l].split = fused_split_uniform(cfg.fused_tz, c->L[l].m[2]);
        } else if (cfg.fused_tz == -1) {
            c->L[l].split = fused_split_uniform(fused_tz_throughput(c->L[l]), c->L[l].m[2]);
        } else if (cfg.autotune) {
            CK(cudaMemsetAsync(c->lb.pdir, 0, sizeof(float) * 3 * c->L[l].nn, c->stream));
            CK(fused_autotune(c, l, c->lb.pdir, c->stream));
        } else {
            c->L[l].split = fused_split(c->L[l], c->num_sms);   // the load model's choice
        }
    }
    if (!ptr_is_device) CK(cudaStreamSynchronize(c->stream));  // host arrays may be released on return
    c->have_images = true;
    return REG_OK;
}

int reg_level_tiling(reg_handle c, int level, int *tz, int *tiles)
{
    if (!c) return set_err(nullptr, REG_ERR_ARG, "reg_level_tiling: NULL handle");
    if (!c->have_images) return set_err(c, REG_ERR_STATE, "reg_level_tiling: no images set");
    if (level < 0 || level >= c->levels)
        return set_err(c, REG_ERR_ARG, "reg_level_tiling: level %d out of range", level);
    int z = 0, n = 0;
    if (use_fused(c, level)) {
        FusedSplit sp;
        int ntx, nty;
        fused_tiling(c->L[level], c->num_sms, &sp, &ntx, &nty);
        z = sp.longest();
        n = ntx * nty * sp.count();
    }
    if (tz) *tz = z;
    if (tiles) *tiles = n;
    return REG_OK;
}

int reg_fused_split_plan(const int dims[3], int num_sms, int split[5], double *model_steps)
{
    if (!dims || !split) return set_err(nullptr, REG_ERR_ARG, "reg_fused_split_plan: NULL argument");
    if (num_sms < 1) return set_err(nullptr, REG_ERR_ARG, "reg_fused_split_plan: num_sms must be >= 1");
    for (int d = 0; d < 3; d++)
        if (dims[d] < 4 || (dims[d] & 1))
            return set_err(nullptr, REG_ERR_ARG, "reg_fused_split_plan: dims[%d] = %d must be even and >= 4", d,
                           dims[d]);
    const FusedSplit sp = fused_split_plan(dims, num_sms, model_steps);
    split[0] = sp.l1;
    split[1] = sp.n1;
    split[2] = sp.l2;
    split[3] = sp.n2;
    split[4] = sp.lr;
    return REG_OK;
}

int reg_fused_tile_shape(int *ox, int *oy, int *ctas_per_sm)
{
    int a = 0, b = 0, c = 0;
    fused_tile_shape(&a, &b, &c);
    if (ox) *ox = a;
    if (oy) *oy = b;
    if (ctas_per_sm) *ctas_per_sm = c;
    return REG_OK;
}

int reg_axis_tables(int m, double h, int n, int *k0, float *w1, int *first, int *cnt, float *w, int max_w,
                    int *needed_w)
{
    if (m < 4 || n < 3 || !(h > 0) || !isfinite(h))
        return set_err(nullptr, REG_ERR_ARG, "reg_axis_tables: need m >= 4, n >= 3 and a finite h > 0");
    const AxisTables a = axis_tables(m, h, m * h / (n - 1), n);
    if (needed_w) *needed_w = a.maxw;
    if (max_w < a.maxw && w)
        return set_err(nullptr, REG_ERR_ARG, "reg_axis_tables: max_w = %d < %d weights per node", max_w, a.maxw);
    for (int i = 0; i < m; i++) {
        if (k0) k0[i] = a.k0[i];
        if (w1) w1[i] = a.w1[i];
    }
    for (int k = 0; k < n; k++) {
        if (first) first[k] = a.first[k];
        if (cnt) cnt[k] = a.cnt[k];
        if (w)
            for (int j = 0; j < max_w; j++) w[(size_t)k * max_w + j] = j < a.maxw ? a.tw[(size_t)k * a.maxw + j] : 0.f;
    }
    return REG_OK;
}

int reg_level_split(reg_handle c, int level, int split[5])
{
    if (!c || !split) return set_err(c, REG_ERR_ARG, "reg_level_split: NULL argument");
    if (!c->have_images) return set_err(c, REG_ERR_STATE, "reg_level_split: no images set");
    if (level < 0 || level >= c->levels)
        return set_err(c, REG_ERR_ARG, "reg_level_split: level %d out of range", level);
    FusedSplit sp;
    if (use_fused(c, level))
        sp = fused_split(c->L[level], c->num_sms);
    split[0] = sp.l1;
    split[1] = sp.n1;
    split[2] = sp.l2;
    split[3] = sp.n2;
    split[4] = sp.lr;
    return REG_OK;
}

int reg_level_info(reg_handle c, int level, int img_dims[3], int node_dims[3], double spacing_mm[3],
                   double node_spacing_mm[3])
{
    if (!c) return set_err(nullptr, REG_ERR_ARG, "reg_level_info: NULL handle");
    if (!c->have_images) return set_err(c, REG_ERR_STATE, "reg_level_info: no images set");
    if (level < 0 || level >= c->levels) return set_err(c, REG_ERR_ARG, "reg_level_info: level %d out of range", level);
    const Level &L = c->L[level];
    for (int d = 0; d < 3; d++) {
        if (img_dims) img_dims[d] = L.m[d];
        if (node_dims) node_dims[d] = L.n[d];
        if (spacing_mm) spacing_mm[d] = L.h[d];
        if (node_spacing_mm) node_spacing_mm[d] = L.H[d];
    }
    return REG_OK;
}

int reg_get_level_image(reg_handle c, int level, int which, float *out, int out_is_device)
{
    if (!c) return set_err(nullptr, REG_ERR_ARG, "reg_get_level_image: NULL handle");
    if (!c->have_images) return set_err(c, REG_ERR_STATE, "reg_get_level_image: no images set");
    if (level < 0 || level >= c->levels || (which != 0 && which != 1) || !out)
        return set_err(c, REG_ERR_ARG, "reg_get_level_image: bad argument");
    const Level &L = c->L[level];
    CK(cudaMemcpyAsync(out, which ? L.T : L.R, sizeof(float) * L.nv,
                       out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return REG_OK;
}

int reg_eval_objective_grad(reg_handle c, int level, const float *u_dev, float *grad_dev, double *J, double *D,
                            double *S)
{
    if (!c) return set_err(nullptr, REG_ERR_ARG, "reg_eval_objective_grad: NULL handle");
    if (!c->have_images) return set_err(c, REG_ERR_STATE, "reg_eval_objective_grad: no images set");
    if (level < 0 || level >= c->levels)
        return set_err(c, REG_ERR_ARG, "reg_eval_objective_grad: level %d out of range", level);
    if (!u_dev || !grad_dev) return set_err(c, REG_ERR_ARG, "reg_eval_objective_grad: NULL vector");
    c->time_ngf = true;
    cudaError_t le = launch_eval(c, level, u_dev, nullptr, nullptr, grad_dev, c->es.scal, -1, c->stream);
    c->time_ngf = false;
    c->kev_valid = le == cudaSuccess;
    CK(le);
    if (J || D || S) {
        double h[3];
        CK(cudaMemcpyAsync(h, c->es.scal, sizeof h, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (J) *J = h[0];
        if (D) *D = h[1];
        if (S) *S = h[2];
        if (!isfinite(h[0])) return set_err(c, REG_ERR_NUMERIC, "reg_eval_objective_grad: J is not finite");
    }
    return REG_OK;
}

int reg_last_ngf_ms(reg_handle c, double *ms)
{
    if (!c || !ms) return set_err(c, REG_ERR_ARG, "reg_last_ngf_ms: NULL argument");
    if (!c->kev_valid) return set_err(c, REG_ERR_STATE, "reg_last_ngf_ms: no evaluation timed yet");
    CK(cudaEventSynchronize(c->kev[1]));
    float f = 0.f;
    CK(cudaEventElapsedTime(&f, c->kev[0], c->kev[1]));
    *ms = f;
    return REG_OK;
}

int reg_prolong(reg_handle c, int level_coarse, const float *uc_dev, float *uf_dev)
{
    if (!c) return set_err(nullptr, REG_ERR_ARG, "reg_prolong: NULL handle");
    if (!c->have_images) return set_err(c, REG_ERR_STATE, "reg_prolong: no images set");
    if (level_coarse < 1 || level_coarse >= c->levels || !uc_dev || !uf_dev)
        return set_err(c, REG_ERR_ARG, "reg_prolong: bad argument");
    CK(launch_prolong(c->L[level_coarse], c->L[level_coarse - 1], uc_dev, uf_dev, c->stream));
    c->launches += 1;
    return REG_OK;
}

int reg_lbfgs_direction(reg_handle c, long long n, int count, const float *S_dev, const float *Y_dev,
                        const float *g_dev, float *p_dev)
{
    if (!c) return set_err(nullptr, REG_ERR_ARG, "reg_lbfgs_direction: NULL handle");
    if (!c->have_images) return set_err(c, REG_ERR_STATE, "reg_lbfgs_direction: no images set");
    if (n <= 0 || count < 0 || count > c->cfg.lbfgs_mem || !g_dev || !p_dev || (count > 0 && (!S_dev || !Y_dev)))
        return set_err(c, REG_ERR_ARG, "reg_lbfgs_direction: bad argument");
    const Level &L = c->L[0];
    double Hmin = fmin(L.H[0], fmin(L.H[1], L.H[2]));
    lbfgs_state_reset_host(c->lb.st_host, c->cfg, 1, Hmin);
    CK(cudaMemcpyAsync(c->lb.st, c->lb.st_host, sizeof(LbfgsState), cudaMemcpyHostToDevice, c->stream));
    CK(lbfgs_direction_standalone(c, n, count, S_dev, Y_dev, g_dev, p_dev, Hmin, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return REG_OK;
}

}  // extern "C"

namespace {

int read_state(reg_ctx *c)
{
    CK(cudaMemcpyAsync(c->lb.st_host, c->lb.st, sizeof(LbfgsState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return REG_OK;
}

// One level of L-BFGS, each step queued by the host; the host reads the
// device state after every line-search trial and every accepted step.
int run_level_host(reg_ctx *c, int level)
{
    LbfgsState *sh = c->lb.st_host;
    int r;
    CK(lbfgs_launch_init(c, level, c->stream));
    if ((r = read_state(c)) != REG_OK) return r;
    // every loop below is bounded by max_iter, max_backtracks and one retry
    const long long guard = 4LL * (sh->max_iter + 1) * (sh->max_bt + 1) + 16;
    long long steps = 0;
    while (!sh->done && sh->iter_continue && steps++ < guard) {
        CK(lbfgs_launch_direction_level(c, level, c->stream));
        do {
            CK(lbfgs_launch_trial(c, level, c->stream));
            if ((r = read_state(c)) != REG_OK) return r;
        } while (sh->ls_continue && steps++ < guard);
        CK(lbfgs_launch_accept_level(c, level, c->stream));
        if ((r = read_state(c)) != REG_OK) return r;
    }
    if (steps >= guard) return set_err(c, REG_ERR_TIMEOUT, "L-BFGS level %d exceeded its step bound", level);
    return REG_OK;
}

// One level as a single graph launch (built on first use); the host reads
// the device state once, after the level.
int run_level_graph(reg_ctx *c, int level)
{
    if (lbfgs_level_loop_ok(c, level)) {   // a small level: one cooperative kernel for its loop
        CK(lbfgs_launch_init(c, level, c->stream));
        CK(lbfgs_launch_level_loop(c, level, c->stream));
        return read_state(c);
    }
    if (!c->iter_graph[level]) {
        cudaError_t e = build_level_graph(c, level, &c->iter_graph[level]);
        if (e != cudaSuccess) {
            c->iter_graph[level] = nullptr;
            return cuda_err(c, e, "building the L-BFGS level graph");
        }
    }
    CK(cudaGraphLaunch(c->iter_graph[level], c->stream));
    int r = read_state(c);
    if (r != REG_OK) return r;
    const LbfgsState *sh = c->lb.st_host;
    const int ek = eval_kernel_count(c, level);
    // init: evaluation + norms (control folded in); per body: direction + accept, plus
    // the p0 redos the IF node ran; per trial: evaluation (Armijo in its final reduction)
    c->launches += (ek + 1) + 2LL * sh->bodies + sh->redos + (long long)ek * (sh->evals - 1);
    return REG_OK;
}

}  // namespace

extern "C" {

int reg_register(reg_handle c, float *u_out, int out_is_device, const float *u_init, reg_stats *st)
{
    auto t0 = std::chrono::steady_clock::now();
    if (!c) return set_err(nullptr, REG_ERR_ARG, "reg_register: NULL handle");
    if (!c->have_images) return set_err(c, REG_ERR_STATE, "reg_register: no images set");
    if (!u_out) return set_err(c, REG_ERR_ARG, "reg_register: NULL u_out");
    const int start = c->cfg.start_level < 0 ? c->levels - 1 : c->cfg.start_level;
    reg_stats local;
    memset(&local, 0, sizeof local);
    local.levels = c->levels;
    LbfgsBuffers &b = c->lb;
    const long long n0 = 3 * c->L[start].nn;
    if (u_init)
        CK(cudaMemcpyAsync(b.u, u_init, sizeof(float) * n0,
                           out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    else
        CK(cudaMemsetAsync(b.u, 0, sizeof(float) * n0, c->stream));
    int status = REG_OK;
    const long long launches0 = c->launches;
    if (!c->lev_ev[0])
        for (int i = 0; i <= REG_MAX_LEVELS; i++)
            CK(cudaEventCreate(&c->lev_ev[i]));
    for (int l = start; l >= 0; l--) {
        const Level &L = c->L[l];
        CK(cudaEventRecord(c->lev_ev[l + 1], c->stream));
        if (l < start) {
            CK(launch_prolong(c->L[l + 1], L, b.u, b.g, c->stream));
            c->launches += 1;
            CK(cudaMemcpyAsync(b.u, b.g, sizeof(float) * 3 * L.nn, cudaMemcpyDeviceToDevice, c->stream));
        }
        double Hmin = fmin(L.H[0], fmin(L.H[1], L.H[2]));
        lbfgs_state_reset_host(b.st_host, c->cfg, c->cfg.max_iter[l], Hmin);
        CK(cudaMemcpyAsync(b.st, b.st_host, sizeof(LbfgsState), cudaMemcpyHostToDevice, c->stream));
        int r = c->cfg.use_graph ? run_level_graph(c, l) : run_level_host(c, l);
        if (r != REG_OK) return r;
        const LbfgsState *sh = b.st_host;
        local.iters[l] = sh->k;
        local.evals[l] = sh->evals;
        local.J[l] = sh->J;
        local.tiling[l] = use_fused(c, l) ? fused_split(c->L[l], c->num_sms).longest() : 0;
        if (sh->status == -5) return set_err(c, REG_ERR_NUMERIC, "reg_register: non-finite J or gradient at level %d", l);
        if (sh->status == -6)
            return set_err(c, REG_ERR_TIMEOUT, "reg_register: level %d exceeded its loop bound", l);
        if (sh->status == -7)
            return set_err(c, REG_ERR_TIMEOUT, "reg_register: a bulk-copy wait of an L-BFGS pass expired at level %d", l);
        local.level_status[l] = sh->status == 1 ? REG_WARN_LINESEARCH : REG_OK;
        if (sh->status == 1) status = REG_WARN_LINESEARCH;
        if (l == 0) {
            local.J_final = sh->J;
            local.D_final = sh->D;
            local.S_final = sh->S;
        }
    }
    CK(cudaEventRecord(c->lev_ev[0], c->stream));
    CK(cudaMemcpyAsync(u_out, b.u, sizeof(float) * 3 * c->L[0].nn,
                       out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int l = start; l >= 0; l--) {   // level l ran from event l + 1 to event l
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->lev_ev[l + 1], c->lev_ev[l]));
        local.level_seconds[l] = 1e-3 * ms;
    }
    local.status = status;
    local.kernel_launches = c->launches - launches0;
    local.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (st) *st = local;
    if (status == REG_WARN_LINESEARCH) set_err(c, status, "reg_register: a line search failed");
    return status;
}

int reg_destroy(reg_handle c)
{
    if (!c) return REG_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_buffers(c);
    for (int i = 0; i <= REG_MAX_LEVELS; i++)
        if (c->lev_ev[i]) cudaEventDestroy(c->lev_ev[i]);
    if (c->ev_side) cudaEventDestroy(c->ev_side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (int i = 0; i < 2; i++)
        if (c->kev[i]) cudaEventDestroy(c->kev[i]);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return REG_OK;
}

const char *reg_last_error(reg_handle c)
{
    if (!c) return g_create_err.c_str();
    return c->err.c_str();
}

}  // extern "C"
