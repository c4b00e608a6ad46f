// Fused objective pass for ratio-2 grids (every image dimension even and
// n_d = m_d / 2 + 1, the default rule): one kernel computes, per voxel,
//   y-hat = P u (Eq. 1), T(x + y-hat) and its interpolant gradient,
//   the NGF residual of Eq. 2 and v = d psi / d grad T,
//   g = adjoint central difference of v, r = g grad T (the chain rule),
// and reduces r to per-tile partial node sums of P^T r (Eq. 3); a second,
// node-parallel kernel adds up the (at most 8) tile partials of each node and
// the curvature gradient.  Nothing per voxel goes to HBM.
//
// Tiling.  A CTA of 32 x 16 threads owns the voxel columns of a 28 x 12 output
// tile plus a 2-voxel halo (the stencil chain T~ -> a -> v -> g reaches two
// voxels), and marches along z through a segment of TZ output planes.  Step s
// computes, in order,
//   A: T~ and grad T at plane zA = z0 - 2 + s   (every thread of the 32 x 16 plane)
//   B: v at plane zA - 1                         (the 30 x 14 inner threads)
//   C: r at plane zA - 2                         (the 28 x 12 output threads)
//   D: P^T of that r plane into node sums        (shuffles in x, shared memory in y,
//                                                  registers in z)
// Neighbours along z live in per-thread registers; along x and y in
// double-buffered shared-memory planes.  With ratio 2 the P weights are 1/4
// and 3/4 and a node gathers voxels 2k-2 .. 2k+1 with weights 1/4, 3/4, 3/4,
// 1/4 per dimension, so an output tile of 28 x 12 x TZ voxels feeds
// 15 x 7 x (TZ/2 + 1) nodes; neighbouring tiles share one node plane per
// dimension and the gather kernel sums them.
#include "internal.h"
#include "ngf_math.cuh"

namespace {

constexpr int BX = 32, BY = 16;            // threads (voxel columns incl. halo)
constexpr int OX = 28, OY = 12;            // output voxels per tile
constexpr int NX = OX / 2 + 1, NY = OY / 2 + 1;   // 15 x 7 node columns per tile
constexpr int NE = 3 * NX * NY;            // partial entries per node plane (315)

struct FusedArgs {
    LevelGeom g;
    const float *T, *R, *ub, *dir;
    const double *t_dev;
    float tau, rho;
    int tz;                 // output planes per z segment (even)
    int ntx, nty, ntz;      // tiles
    float *part;            // [tile][TZ/2 + 1][NE]
    double *partials;       // D block partials
};

// node value at the trial point u + t dir (HAS_DIR) or u
template <bool HAS_DIR>
__device__ __forceinline__ float nval(const float *__restrict__ u, const float *__restrict__ d, float t, int k)
{
    float v = __ldg(u + k);
    if (HAS_DIR)
        v = fmaf(t, __ldg(d + k), v);
    return v;
}

// displacement plane K of this thread's column: value at the first node and
// the bilinear interpolation of the in-plane node differences to it
template <bool HAS_DIR>
__device__ __forceinline__ void load_node_plane(const FusedArgs &a, int kx, int ky, int K, float wx, float wy,
                                                float t, float U[3], float Bd[3])
{
    const LevelGeom &g = a.g;
    if (K < 0 || K >= g.n[2]) {
        U[0] = U[1] = U[2] = 0.f;
        Bd[0] = Bd[1] = Bd[2] = 0.f;
        return;
    }
    const int sy = g.n[0];
    const int b = kx + sy * (ky + g.n[1] * K);
    const int nn = (int)g.nn;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float *u = a.ub + c * nn;
        const float *d = a.dir + (HAS_DIR ? c * nn : 0);
        float u00 = nval<HAS_DIR>(u, d, t, b);
        float d10 = nval<HAS_DIR>(u, d, t, b + 1) - u00;
        float d01 = nval<HAS_DIR>(u, d, t, b + sy) - u00;
        float d11 = nval<HAS_DIR>(u, d, t, b + sy + 1) - u00;
        U[c] = u00;
        Bd[c] = lerpf(wx * d10, lerpf(d01, d11, wx), wy);
    }
}

template <bool HAS_DIR>
__global__ void __launch_bounds__(BX * BY, 1) k_ngf_fused(FusedArgs a)
{
    __shared__ float sT[2][BY][BX];      // T~ planes (double buffered)
    __shared__ float sR[2][BY][BX];      // R planes
    __shared__ float sVx[2][BY][BX];     // v_x planes
    __shared__ float sVy[2][BY][BX];     // v_y planes
    __shared__ float sRed[BY][NX][3];    // x-reduced r rows
    __shared__ double sm[BX * BY / 32];

    const LevelGeom &g = a.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int tile_x = blockIdx.x, tile_y = blockIdx.y, tile_z = blockIdx.z;
    const int x = tile_x * OX - 2 + tx;
    const int y = tile_y * OY - 2 + ty;
    const int z0 = tile_z * a.tz;
    const int mx = g.m[0], my = g.m[1], mz = g.m[2];
    const bool col_in = x >= 0 && x < mx && y >= 0 && y < my;
    const bool b_thr = tx >= 1 && tx < BX - 1 && ty >= 1 && ty < BY - 1;
    const bool c_thr = tx >= 2 && tx < BX - 2 && ty >= 2 && ty < BY - 2;
    const float t = HAS_DIR ? (float)__ldg(a.t_dev) : 0.f;

    // ratio 2: voxel i lies between nodes i/2 and i/2 + 1, weight of the second 1/4 or 3/4
    const int kx = x >> 1, ky = y >> 1;
    const float wx = (x & 1) ? 0.75f : 0.25f, wy = (y & 1) ? 0.75f : 0.25f;

    // per-column state
    float Ulo[3], Blo[3], Uhi[3], Bhi[3];
    int Klo = (z0 - 2) >> 1;
    if (col_in) {
        load_node_plane<HAS_DIR>(a, kx, ky, Klo, wx, wy, t, Ulo, Blo);
        load_node_plane<HAS_DIR>(a, kx, ky, Klo + 1, wx, wy, t, Uhi, Bhi);
    }
    float Tq0 = 0.f, Tq1 = 0.f, Tq2 = 0.f;    // T~ at zA-2, zA-1, zA
    float Rq0 = 0.f, Rq1 = 0.f, Rq2 = 0.f;    // R at zA-2, zA-1, zA
    float vz0 = 0.f, vz1 = 0.f, vz2 = 0.f;    // v_z at zA-3, zA-2, zA-1
    float gq[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};  // grad T at zA-2, zA-1, zA
    float acc_lo = 0.f, acc_hi = 0.f;         // z accumulation of partial entry `tid`
    KahanF psi_sum;
    const float hx = 0.5f * g.ih[0], hy = 0.5f * g.ih[1], hz = 0.5f * g.ih[2];
    const float half_hbar = 0.5f * g.hbar;
    const size_t tile_lin = (size_t)tile_x + (size_t)a.ntx * (tile_y + (size_t)a.nty * tile_z);
    float *part_tile = a.part + tile_lin * (size_t)(a.tz / 2 + 1) * NE;

    const int nsteps = a.tz + 4;
    for (int s = 0; s < nsteps; s++) {
        const int zA = z0 - 2 + s;
        const int buf = s & 1;
        // ---- A: T~ and grad T at (x, y, zA); R at (x, y, zA)
        {
            // advance the node planes when zA enters a new node interval
            if (s > 0 && !(zA & 1)) {
                Klo++;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    Ulo[c] = Uhi[c];
                    Blo[c] = Bhi[c];
                }
                if (col_in)
                    load_node_plane<HAS_DIR>(a, kx, ky, Klo + 1, wx, wy, t, Uhi, Bhi);
            }
            float val = 0.f, gr[3] = {0.f, 0.f, 0.f}, rv = 0.f;
            if (col_in && zA >= 0 && zA < mz) {
                const float wz = (zA & 1) ? 0.75f : 0.25f;
                int cc[3];
                float ff[3];
                bool ok[3];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    // y-hat = U_lo + lerp(B_lo, (U_hi - U_lo) + B_hi, wz)
                    float delta = lerpf(Blo[c], (Uhi[c] - Ulo[c]) + Bhi[c], wz);
                    int i = c == 0 ? x : (c == 1 ? y : zA);
                    sample_coord(i, Ulo[c], delta, g.h[c], g.ih[c], cc[c], ff[c], ok[c]);
                }
                interp_value_grad(a.T, mx, my, mz, cc, ff, ok[0] && ok[1] && ok[2], g.ih, val, gr);
                rv = __ldg(a.R + (x + mx * (y + my * zA)));
            }
            Tq0 = Tq1;
            Tq1 = Tq2;
            Tq2 = val;
            Rq0 = Rq1;
            Rq1 = Rq2;
            Rq2 = rv;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                gq[0][c] = gq[1][c];
                gq[1][c] = gq[2][c];
                gq[2][c] = gr[c];
            }
            sT[buf][ty][tx] = val;
            sR[buf][ty][tx] = rv;
        }
        __syncthreads();
        // ---- B: v at (x, y, zB = zA - 1)
        const int zB = zA - 1;
        {
            float v[3] = {0.f, 0.f, 0.f};
            if (b_thr && s >= 1) {
                const int bb = buf ^ 1;   // plane zB was written at step s - 1
                bool interior = col_in && x >= 1 && x <= mx - 2 && y >= 1 && y <= my - 2 && zB >= 1 && zB <= mz - 2;
                if (interior) {
                    float av[3], bv[3];
                    av[0] = (sT[bb][ty][tx + 1] - sT[bb][ty][tx - 1]) * hx;
                    av[1] = (sT[bb][ty + 1][tx] - sT[bb][ty - 1][tx]) * hy;
                    av[2] = (Tq2 - Tq0) * hz;
                    bv[0] = (sR[bb][ty][tx + 1] - sR[bb][ty][tx - 1]) * hx;
                    bv[1] = (sR[bb][ty + 1][tx] - sR[bb][ty - 1][tx]) * hy;
                    bv[2] = (Rq2 - Rq0) * hz;
                    float psi = ngf_residual(av, bv, a.tau, a.rho, v);
                    if (c_thr && zB >= z0 && zB < z0 + a.tz)
                        psi_sum.add(psi);
                }
            }
            if (b_thr) {
                sVx[buf][ty][tx] = v[0];
                sVy[buf][ty][tx] = v[1];
            }
            vz0 = vz1;
            vz1 = vz2;
            vz2 = v[2];
        }
        __syncthreads();
        // ---- C: r at (x, y, zC = zA - 2); D: x reduction of the r row
        const int zC = zA - 2;
        const int lz = zC - z0;          // output plane index inside the segment
        const bool c_plane = lz >= 0 && lz < a.tz;
        if (c_plane) {
            float r[3] = {0.f, 0.f, 0.f};
            if (c_thr && col_in && zC < mz) {
                const int vb = buf ^ 1;   // v of plane zC was written at step s - 1
                float gs = (sVx[vb][ty][tx - 1] - sVx[vb][ty][tx + 1]) * hx +
                           (sVy[vb][ty - 1][tx] - sVy[vb][ty + 1][tx]) * hy + (vz0 - vz2) * hz;
                float gj = half_hbar * gs;
                r[0] = gj * gq[0][0];
                r[1] = gj * gq[0][1];
                r[2] = gj * gq[0][2];
            }
            // node column j (0..14) of this row gathers threads 2j .. 2j+3 with 1/4, 3/4, 3/4, 1/4
#pragma unroll
            for (int c = 0; c < 3; c++) {
                float r1 = __shfl_down_sync(0xffffffffu, r[c], 1);
                float r2 = __shfl_down_sync(0xffffffffu, r[c], 2);
                float r3 = __shfl_down_sync(0xffffffffu, r[c], 3);
                // written nodes have tx = 2j <= 28, so lanes tx + 1 .. tx + 3 exist
                if (!(tx & 1) && (tx >> 1) < NX)
                    sRed[ty][tx >> 1][c] = 0.25f * (r[c] + r3) + 0.75f * (r1 + r2);
            }
        }
        __syncthreads();
        if (c_plane) {
            // y reduction of entry tid = (c, jy, jx) and accumulation along z
            if (tid < NE) {
                const int c = tid / (NX * NY), rem = tid % (NX * NY), jy = rem / NX, jx = rem % NX;
                const int r0 = 2 * jy;
                float v = 0.25f * sRed[r0][jx][c] + 0.75f * (sRed[r0 + 1][jx][c] + sRed[r0 + 2][jx][c]) +
                          0.25f * sRed[r0 + 3][jx][c];
                if (!(lz & 1)) {
                    acc_lo = fmaf(0.75f, v, acc_lo);
                    acc_hi = fmaf(0.25f, v, acc_hi);
                } else {
                    acc_lo = fmaf(0.25f, v, acc_lo);
                    acc_hi = fmaf(0.75f, v, acc_hi);
                    // node plane lz / 2 of the segment is complete
                    part_tile[(size_t)(lz >> 1) * NE + tid] = acc_lo;
                    acc_lo = acc_hi;
                    acc_hi = 0.f;
                }
                if (lz == a.tz - 1)
                    part_tile[(size_t)(a.tz >> 1) * NE + tid] = acc_lo;
            }
        }
        // the next step's writes to sRed follow two more barriers
    }
    double ssum = block_sum_to_f64(psi_sum.s, sm);
    if (tid == 0)
        a.partials[(size_t)blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z)] = ssum;
}

// grad J at node k = sum of the tile partials that contain k (P^T r) plus
// alpha hbar_y L^T w (curvature), one thread per node, 3 components.
__global__ void __launch_bounds__(256) k_gather_grad(LevelGeom g, const float *__restrict__ part, int tz, int ntx,
                                                     int nty, int ntz, const float *__restrict__ w, float alpha_hy,
                                                     float *__restrict__ grad)
{
    int kx = blockIdx.x * blockDim.x + threadIdx.x;
    int ky = blockIdx.y * blockDim.y + threadIdx.y;
    int kz = blockIdx.z;
    if (kx >= g.n[0] || ky >= g.n[1])
        return;
    const int hz = tz / 2;
    const size_t plane_stride = (size_t)(hz + 1) * NE;
    float s[3] = {0.f, 0.f, 0.f};
    // candidate tiles per dimension: t = k / step and t - 1, local index k - step * t in [0, step]
    for (int dz = 0; dz < 2; dz++) {
        int tzi = kz / hz - dz;
        int jz = kz - hz * tzi;
        if (tzi < 0 || tzi >= ntz || jz > hz)
            continue;
        for (int dy = 0; dy < 2; dy++) {
            int tyi = ky / (NY - 1) - dy;
            int jy = ky - (NY - 1) * tyi;
            if (tyi < 0 || tyi >= nty || jy > NY - 1)
                continue;
            for (int dx = 0; dx < 2; dx++) {
                int txi = kx / (NX - 1) - dx;
                int jx = kx - (NX - 1) * txi;
                if (txi < 0 || txi >= ntx || jx > NX - 1)
                    continue;
                size_t tile = (size_t)txi + (size_t)ntx * (tyi + (size_t)nty * tzi);
                const float *p = part + tile * plane_stride + (size_t)jz * NE + jy * NX + jx;
                s[0] += __ldg(p);
                s[1] += __ldg(p + NX * NY);
                s[2] += __ldg(p + 2 * NX * NY);
            }
        }
    }
    size_t k = kx + (size_t)g.n[0] * (ky + (size_t)g.n[1] * kz);
    size_t st[3] = {1, (size_t)g.n[0], (size_t)g.n[0] * g.n[1]};
    int j[3] = {kx, ky, kz};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float *wc = w + c * g.nn;
        float w0 = __ldg(wc + k);
        float l = 0.f;
#pragma unroll
        for (int e = 0; e < 3; e++) {
            float lo = j[e] > 0 ? __ldg(wc + k - st[e]) : 0.f;
            float hi = j[e] < g.n[e] - 1 ? __ldg(wc + k + st[e]) : 0.f;
            l = fmaf(lo + hi - 2.f * w0, g.iH2[e], l);
        }
        grad[c * g.nn + k] = fmaf(alpha_hy, l, s[c]);
    }
}

}  // namespace

bool fused_eligible(const Level &L)
{
    for (int d = 0; d < 3; d++)
        if ((L.m[d] & 1) || L.n[d] != L.m[d] / 2 + 1)
            return false;
    return true;
}

// z segment length: even, 8 .. 64, aiming at >= 2 CTAs per SM
int fused_tz(const Level &L, int num_sms)
{
    long long cols = (long long)((L.m[0] + OX - 1) / OX) * ((L.m[1] + OY - 1) / OY);
    int tz = 64;
    while (tz > 8 && cols * ((L.m[2] + tz - 1) / tz) < 2LL * num_sms)
        tz /= 2;
    return tz;
}

void fused_grid(const Level &L, int tz, int &ntx, int &nty, int &ntz)
{
    ntx = (L.m[0] + OX - 1) / OX;
    nty = (L.m[1] + OY - 1) / OY;
    ntz = (L.m[2] + tz - 1) / tz;
}

size_t fused_part_floats(const Level &L, int num_sms)
{
    int tz = fused_tz(L, num_sms), ntx, nty, ntz;
    fused_grid(L, tz, ntx, nty, ntz);
    return (size_t)ntx * nty * ntz * (tz / 2 + 1) * NE;
}

cudaError_t launch_ngf_fused(reg_ctx *c, int level, const float *ub, const float *dir, const double *t_dev,
                             float *grad, double *partials, int *n_partials, cudaStream_t s)
{
    (void)grad;
    const Level &L = c->L[level];
    FusedArgs a;
    a.g = L.geom();
    a.T = L.T;
    a.R = L.R;
    a.ub = ub;
    a.dir = dir;
    a.t_dev = t_dev;
    a.tau = (float)c->cfg.tau;
    a.rho = (float)c->cfg.rho;
    a.tz = fused_tz(L, c->num_sms);
    fused_grid(L, a.tz, a.ntx, a.nty, a.ntz);
    a.part = c->es.part;
    a.partials = partials;
    dim3 blk(BX, BY, 1), grd(a.ntx, a.nty, a.ntz);
    if (dir)
        k_ngf_fused<true><<<grd, blk, 0, s>>>(a);
    else
        k_ngf_fused<false><<<grd, blk, 0, s>>>(a);
    *n_partials = a.ntx * a.nty * a.ntz;
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_gather_grad(reg_ctx *c, int level, const float *w, float alpha_hy, float *grad, cudaStream_t s)
{
    const Level &L = c->L[level];
    int tz = fused_tz(L, c->num_sms), ntx, nty, ntz;
    fused_grid(L, tz, ntx, nty, ntz);
    dim3 blk(32, 8, 1);
    dim3 gn((L.n[0] + 31) / 32, (L.n[1] + 7) / 8, L.n[2]);
    k_gather_grad<<<gn, blk, 0, s>>>(L.geom(), c->es.part, tz, ntx, nty, ntz, w, alpha_hy, grad);
    c->launches += 1;
    return cudaGetLastError();
}
