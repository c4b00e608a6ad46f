// reg_eval_objective_grad_noalloc: one objective + gradient evaluation whose
// working memory is a fixed array in the library's device image instead of
// memory allocated per call.
//
// Who needs this: callers that are not allowed to allocate device memory at
// call time - code that runs inside a host framework which owns all device
// memory through its own pool and budget (a cudaMalloc behind its back can
// exceed the budget or fragment the pool), and latency-bound loops that must
// not take the driver's allocation path (cudaMalloc and cudaFree may
// synchronise the device).  They pass their own input and output buffers; the
// intermediate sums live in g_noalloc_scratch below.
//
// The array is a file-scope __device__ variable, so every GPU that loads this
// library holds it until the process exits.  Host code cannot use the name
// g_noalloc_scratch as a device address (it names a host-side stand-in), so
// the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current, and caches it with the
// id of the device's context: after a device reset the context is new, and
// the next call repeats the set-up.
#include <cuda.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "internal.h"

// explicit-buffer launchers (k_ngf_fused.cu, k_curv.cu)
void fused_layout_dims(const int m[3], int num_sms, int *tz, int *tiles, size_t *part_floats);
cudaError_t fused_set_smem_limit();
cudaError_t launch_ngf_fused_raw(const LevelGeom &g, const float *T, const float *R, const float *u, float tau,
                                 float rho, int num_sms, float *part, double *partials, float *w, cudaStream_t s);
cudaError_t launch_gather_grad_raw(const LevelGeom &g, const float *part, int num_sms, const float *w,
                                   float alpha_hy, float *grad, cudaStream_t s);
cudaError_t launch_finalize_raw(const double *pD, int nD, const double *pS, int nS, double hbar_half, double alpha,
                                double hy_half, double *scal, cudaStream_t s);
int set_err(reg_ctx *c, int code, const char *fmt, ...);

namespace {

// Capacities of the shared scratch (bytes in parentheses):
//   tile partial sums of P^T r : 2^22 floats      (16 MiB)
//   curvature Laplacian w      : 2^20 floats      (4 MiB)
//   block partial sums         : 2^16 doubles     (512 KiB)
// 256^3 images do not fit; a 128^3 pair needs at most 2.3 M + 0.82 M floats
// and a few thousand doubles, and the Laplacian w limits the size to about
// 136^3 (which needs at most 2.6 M partial floats).
constexpr size_t CAP_PART = size_t(1) << 22;
constexpr size_t CAP_W = size_t(1) << 20;
constexpr size_t CAP_PARTIALS = size_t(1) << 16;
constexpr size_t OFFB_PART = 0;
constexpr size_t OFFB_W = OFFB_PART + CAP_PART * sizeof(float);
constexpr size_t OFFB_PARTIALS = OFFB_W + CAP_W * sizeof(float);
constexpr size_t SCRATCH_BYTES = OFFB_PARTIALS + CAP_PARTIALS * sizeof(double);

constexpr int MAX_DEVICES = 64;
// longest image side (voxels); with at least 4 voxels in the other two
// dimensions the Laplacian's capacity allows up to about 77000
constexpr int MAX_DIM = 4096;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

struct DeviceSetup {
    void *scratch = nullptr;   // device address of g_noalloc_scratch on that device
    int num_sms = 0;
    unsigned long long ctx_id = 0;   // context the address and the attribute belong to
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[MAX_DEVICES];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (0: none current or the
// driver lacks the query).  Driver entry points come through the runtime, so
// the library needs no link against the driver library.
unsigned long long current_ctx_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(a);
            get_id = reinterpret_cast<CtxGetIdFn>(b);
        }
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Once per device and context, with that device current: the device address
// of the scratch array, the SM count, and the fused kernel's shared-memory
// limit.
int device_setup(int dev, DeviceSetup *out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &d = g_setup[dev];
    const unsigned long long ctx = current_ctx_id();
    if (!d.scratch || ctx == 0 || ctx != d.ctx_id) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess)
            return set_err(nullptr, REG_ERR_CUDA, "reg_eval_objective_grad_noalloc: cudaGetSymbolAddress: %s",
                           cudaGetErrorString(e));
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = fused_set_smem_limit();
        if (e != cudaSuccess)
            return set_err(nullptr, REG_ERR_CUDA, "reg_eval_objective_grad_noalloc: device set-up: %s",
                           cudaGetErrorString(e));
        d.num_sms = sms;
        d.scratch = ptr;
        d.ctx_id = current_ctx_id();   // the look-up above made the context current if none was
    }
    *out = d;
    return REG_OK;
}

}  // namespace

extern "C" int reg_eval_objective_grad_noalloc(const float *R, const float *T, const int dims[3],
                                               const double spacing_mm[3], const float *u, float *grad,
                                               double tau, double rho, double alpha, double *jds,
                                               void *cuda_stream)
{
    const char *fn = "reg_eval_objective_grad_noalloc";
    if (!R || !T || !dims || !spacing_mm || !u || !grad || !jds)
        return set_err(nullptr, REG_ERR_ARG, "%s: NULL argument", fn);
    if (!(tau > 0) || !(rho > 0) || !(alpha >= 0))
        return set_err(nullptr, REG_ERR_ARG, "%s: need tau > 0, rho > 0, alpha >= 0", fn);
    if (reinterpret_cast<uintptr_t>(R) % 8 != 0)   // R is read two voxels at a time
        return set_err(nullptr, REG_ERR_ARG, "%s: R must be 8-byte aligned", fn);
    LevelGeom g;
    memset(&g, 0, sizeof g);
    double H[3];
    for (int d = 0; d < 3; d++) {
        if (dims[d] < 4 || (dims[d] & 1))
            return set_err(nullptr, REG_ERR_ARG, "%s: dims[%d] = %d must be even and >= 4", fn, d, dims[d]);
        if (!(spacing_mm[d] > 0) || !isfinite(spacing_mm[d]))
            return set_err(nullptr, REG_ERR_ARG, "%s: spacing[%d] must be finite and > 0", fn, d);
        g.m[d] = dims[d];
        g.n[d] = dims[d] / 2 + 1;
        H[d] = dims[d] * spacing_mm[d] / (g.n[d] - 1);
        g.h[d] = (float)spacing_mm[d];
        g.ih[d] = (float)(1.0 / spacing_mm[d]);
        g.iH2[d] = (float)(1.0 / (H[d] * H[d]));
    }
    g.hbar = (float)(spacing_mm[0] * spacing_mm[1] * spacing_mm[2]);
    g.hbar_y = (float)(H[0] * H[1] * H[2]);
    g.nv = (long long)g.m[0] * g.m[1] * g.m[2];
    g.nn = (long long)g.n[0] * g.n[1] * g.n[2];

    // the cheap bound first: the node Laplacian w takes 3 floats per node, and
    // each dimension is capped, so the split search below only sees sizes that
    // fit (about 138 voxels per dimension for a cube)
    const size_t w_floats = 3 * (size_t)g.nn;
    if (w_floats > CAP_W || g.m[0] > MAX_DIM || g.m[1] > MAX_DIM || g.m[2] > MAX_DIM)
        return set_err(nullptr, REG_ERR_ARG,
                       "%s: %dx%dx%d needs %zu node floats (max %zu, at most %d voxels per dimension); use a "
                       "handle (reg_create) for larger images",
                       fn, g.m[0], g.m[1], g.m[2], w_floats, CAP_W, MAX_DIM);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return set_err(nullptr, REG_ERR_CUDA, "%s: cudaGetDevice: %s", fn, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES)
        return set_err(nullptr, REG_ERR_ARG, "%s: device %d beyond %d", fn, dev, MAX_DEVICES);
    DeviceSetup ds;
    int r = device_setup(dev, &ds);
    if (r != REG_OK)
        return r;

    // sizes this geometry needs, against the fixed capacities
    int tz = 0, tiles = 0;
    size_t part_floats = 0;
    fused_layout_dims(g.m, ds.num_sms, &tz, &tiles, &part_floats);
    const int nS = tiles;   // the fused pass writes a D and an S partial per tile
    const size_t partials = (size_t)tiles + (size_t)nS;
    if (part_floats > CAP_PART || w_floats > CAP_W || partials > CAP_PARTIALS)
        return set_err(nullptr, REG_ERR_ARG,
                       "%s: %dx%dx%d needs %zu partial floats (max %zu), %zu node floats (max %zu), %zu block "
                       "sums (max %zu); use a handle (reg_create) for larger images",
                       fn, g.m[0], g.m[1], g.m[2], part_floats, CAP_PART, w_floats, CAP_W, partials, CAP_PARTIALS);

    unsigned char *base = static_cast<unsigned char *>(ds.scratch);
    float *part = reinterpret_cast<float *>(base + OFFB_PART);
    float *w = reinterpret_cast<float *>(base + OFFB_W);
    double *pD = reinterpret_cast<double *>(base + OFFB_PARTIALS);
    double *pS = pD + tiles;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // every scratch word read below is written first in the same call, so
    // nothing has to be cleared between calls; the fused pass also writes the
    // curvature Laplacian w and the S partials (after the D partials)
    e = launch_ngf_fused_raw(g, T, R, u, (float)tau, (float)rho, ds.num_sms, part, pD, w, s);
    if (e == cudaSuccess)
        e = launch_gather_grad_raw(g, part, ds.num_sms, w, (float)(alpha * H[0] * H[1] * H[2]), grad, s);
    if (e == cudaSuccess)
        e = launch_finalize_raw(pD, tiles, pS, nS, 0.5 * (double)spacing_mm[0] * spacing_mm[1] * spacing_mm[2],
                                alpha, 0.5 * H[0] * H[1] * H[2], jds, s);
    if (e != cudaSuccess)
        return set_err(nullptr, REG_ERR_CUDA, "%s: launch: %s", fn, cudaGetErrorString(e));
    return REG_OK;
}
