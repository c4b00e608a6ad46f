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
// voxels), and marches along z through a segment of TZ output planes.  With
// ratio 2 the P weights are 1/4 and 3/4 and a node gathers voxels 2k-2 .. 2k+1
// with weights 1/4, 3/4, 3/4, 1/4 per dimension, so an output tile of
// 28 x 12 x TZ voxels feeds 15 x 7 x (TZ/2 + 1) nodes; neighbouring tiles share
// one node plane per dimension and the gather kernel sums them.
//
// Pipeline.  Step s (zA = z0 - 2 + 2 s, even) handles two planes, exactly one
// node interval, between two barriers:
//   A-finish zA, zA+1   : interpolate T on both planes from the corners loaded
//                         last step
//   A-issue  zA+2, zA+3 : P on the next node interval, the coordinates of both
//                         planes, loads of their 2 x 8 corners and of R into
//                         registers (used one step later); cp.async of the
//                         node-plane tile two intervals ahead
//   B  zA-3, zA-2       : v from T~ and R planes zA-4 .. zA-1
//   C  zA-6, zA-5       : r from v planes zA-7 .. zA-4; x reduction by warp shuffles
//   D  zA-8, zA-7       : y reduction of last step's rows, accumulation of one
//                         node interval along z
// Every phase reads only what earlier steps wrote, so one barrier per step
// suffices; the global loads of two planes overlap a whole step of compute, and
// the two planes of each phase are independent work the compiler interleaves.
#include <array>
#include <map>
#include <mutex>

#include "batch.h"
#include "internal.h"
#include "lbfgs_control.cuh"
#include "ngf_math.cuh"

namespace {

constexpr int BX = 32, BY = 16;                   // threads (voxel columns incl. halo)
constexpr int OX = 28, OY = 12;                   // output voxels per tile
constexpr int NX = OX / 2 + 1, NY = OY / 2 + 1;   // 15 x 7 node columns per tile
constexpr int NE = 3 * NX * NY;                   // partial entries per node plane (315)
constexpr int PLANE = BX * BY;                    // floats of one shared plane
constexpr int TNX = BX / 2 + 1, TNY = BY / 2 + 1; // node tile of the columns: 17 x 9
constexpr int TNP = 3 * TNY * TNX;                // floats of one node plane tile per array

// shared layout (floats); the plane rings hold 8 planes (slot z & 7)
constexpr int OFF_T = 0;                          // T~ ring [8][PLANE]
constexpr int OFF_R = OFF_T + 8 * PLANE;          // R ring [8][PLANE]
constexpr int OFF_V = OFF_R + 8 * PLANE;          // v ring [8][3][PLANE]
constexpr int OFF_G = OFF_V + 24 * PLANE;         // grad T ring [8][3][PLANE]
constexpr int RED_PLANE = BY * NX * 3;            // x-reduced rows of one plane
constexpr int OFF_RED = OFF_G + 24 * PLANE;       // x-reduced rows [2 steps][2 planes][BY][NX][3]
constexpr int OFF_N = OFF_RED + 4 * RED_PLANE;    // node planes [4][2][TNP] (u, dir)
constexpr int SMEM_FLOATS = OFF_N + 4 * 2 * TNP;
constexpr size_t SMEM_BYTES = sizeof(float) * SMEM_FLOATS;


__device__ __forceinline__ void cp_async4(float *smem_dst, const float *gsrc, bool valid)
{
    unsigned saddr = (unsigned)__cvta_generic_to_shared(smem_dst);
    int src_size = valid ? 4 : 0;   // 0: no bytes read, the word is zero-filled
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(saddr), "l"(gsrc), "r"(src_size)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One thread's share of the cooperative copy of a node plane (u and, with a
// direction, dir) of the CTA's 17 x 9 node tile: entries tid and tid + PLANE.
// The in-plane offsets do not change along z, so they are computed once.
struct NodeCopy {
    const float *src[2];   // node (kx, ky, plane 0) of the entry's component and array
    int dst[2];            // offset inside a ring slot
    bool in[2];            // node column inside the grid
};

template <bool HAS_DIR>
__device__ __forceinline__ NodeCopy node_copy_setup(const FusedArgs &a, int kx0, int ky0, int tid)
{
    const LevelGeom &g = a.g;
    const int nn = (int)g.nn, total = (HAS_DIR ? 2 : 1) * TNP;
    NodeCopy nc;
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int e = tid + q * PLANE;
        const int arr = e / TNP, r = e - arr * TNP;
        const int c = r / (TNY * TNX), r2 = r - c * (TNY * TNX);
        const int ly = r2 / TNX, lx = r2 - ly * TNX;
        const int kx = kx0 + lx, ky = ky0 + ly;
        nc.in[q] = e < total && kx >= 0 && kx < g.n[0] && ky >= 0 && ky < g.n[1];
        nc.dst[q] = e < total ? e : -1;
        nc.src[q] = nc.in[q] ? (arr ? a.dir : a.ub) + c * nn + (kx + g.n[0] * ky) : a.ub;
    }
    return nc;
}

// copy node plane K into ring slot K % 4; nodes outside the grid read as zero
__device__ __forceinline__ void issue_node_plane(const NodeCopy &nc, float *sm, int K, int nz, int plane_stride)
{
    float *dst = sm + OFF_N + (K & 3) * 2 * TNP;
    const bool kin = K >= 0 && K < nz;
#pragma unroll
    for (int q = 0; q < 2; q++)
        if (nc.dst[q] >= 0) {
            const bool in = kin && nc.in[q];
            cp_async4(dst + nc.dst[q], in ? nc.src[q] + (size_t)plane_stride * K : nc.src[q], in);
        }
}

// displacement plane K of a column from the shared node tile: the value at the
// first node (U) and the bilinear interpolation of the in-plane differences (Bd)
template <bool HAS_DIR>
__device__ __forceinline__ void column_plane(const float *sm, int K, int lkx, int lky, float wx, float wy, float t,
                                             float U[3], float Bd[3])
{
    const float *nu = sm + OFF_N + (K & 3) * 2 * TNP;
    const float *np = nu + TNP;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int o = c * (TNY * TNX) + lky * TNX + lkx;
        float u00 = nu[o], u10 = nu[o + 1], u01 = nu[o + TNX], u11 = nu[o + TNX + 1];
        if (HAS_DIR) {   // trial point u + t dir, the same fmaf as the accepted update
            u00 = fmaf(t, np[o], u00);
            u10 = fmaf(t, np[o + 1], u10);
            u01 = fmaf(t, np[o + TNX], u01);
            u11 = fmaf(t, np[o + TNX + 1], u11);
        }
        U[c] = u00;
        Bd[c] = lerpf(wx * (u10 - u00), lerpf(u01 - u00, u11 - u00, wx), wy);
    }
}

// image element loads: FP32, or BF16 widened to FP32 (all arithmetic is FP32)
__device__ __forceinline__ float ldimg(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldimg(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }

template <typename IMG>
__device__ __forceinline__ float ldimg_zero_ext(const IMG *T, int mx, int my, int mz, int x, int y, int z)
{
    bool in = (unsigned)x < (unsigned)mx && (unsigned)y < (unsigned)my && (unsigned)z < (unsigned)mz;
    return in ? ldimg(T + (x + mx * (y + my * z))) : 0.f;
}

// One output tile (tile_x, tile_y, tile_z) of the fused pass; sm is the CTA's
// dynamic shared memory (SMEM_BYTES).
template <bool HAS_DIR, typename IMG>
__device__ __forceinline__ void fused_tile(const FusedArgs &a, int tile_x, int tile_y, int tile_z, float *sm)
{
    const LevelGeom &g = a.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int x0 = tile_x * OX, y0 = tile_y * OY, z0 = tile_z * a.tz;
    const int x = x0 - 2 + tx, y = y0 - 2 + ty;
    const int mx = g.m[0], my = g.m[1], mz = g.m[2];
    const int sxy = mx * my;
    const bool col_in = x >= 0 && x < mx && y >= 0 && y < my;
    const float t = HAS_DIR ? (float)__ldg(a.t_dev) : 0.f;
    // ratio 2: voxel i lies between nodes i/2 and i/2 + 1, weight of the second 1/4 or 3/4
    const int lkx = tx >> 1, lky = ty >> 1;           // node of the column inside the tile
    const int kx0 = (x0 >> 1) - 1, ky0 = (y0 >> 1) - 1;
    const float wx = (x & 1) ? 0.75f : 0.25f, wy = (y & 1) ? 0.75f : 0.25f;
    const float hx = 0.5f * g.ih[0], hy = 0.5f * g.ih[1], hz = 0.5f * g.ih[2];
    const float half_hbar = 0.5f * g.hbar;
    const int zend = z0 + a.tz;                       // first plane after the segment's output planes
    const size_t tile_lin = (size_t)tile_x + (size_t)a.ntx * (tile_y + (size_t)a.nty * tile_z);
    float *part_tile = a.part + tile_lin * (size_t)(a.tz / 2 + 1) * NE;
    const NodeCopy nc = node_copy_setup<HAS_DIR>(a, kx0, ky0, tid);
    const int node_plane = g.n[0] * g.n[1];
    const IMG *Tim = static_cast<const IMG *>(a.T);
    const IMG *Rcol = static_cast<const IMG *>(a.R) + (col_in ? x + mx * y : 0);
    // output columns and the rows phases B and C run on
    const bool rowB = ty >= 1 && ty < BY - 1, rowC = ty >= 2 && ty < BY - 2;
    const bool colB = tx >= 1 && tx < BX - 1, colC = tx >= 2 && tx < BX - 2;
    const bool intxy = col_in && x >= 1 && x <= mx - 2 && y >= 1 && y <= my - 2;
    // phase D: partial entry tid = (component, node row jy, node column jx)
    const bool dD = tid < NE;
    const int dc = tid / (NX * NY), drem = tid - dc * (NX * NY), djy = drem / NX, djx = drem - djy * NX;
    const int dofs = ((2 * djy) * NX + djx) * 3 + dc;

    float Uhi[3], Bhi[3];                             // node plane of the interval's upper end, this column
    float pc[2][8];                                   // corners of the next two planes, loaded a step ahead
    float fr[2][3];                                   // their fractions
    float rnext[2];                                   // R of the next two planes
    float acc_lo = 0.f;                               // node plane of the interval's lower end (entry tid)
    KahanF psi_sum;

    // rows of the x-reduction buffers that no output row writes stay zero
    for (int e = tid; e < 4 * RED_PLANE; e += PLANE)
        sm[OFF_RED + e] = 0.f;

    // ---- A-issue: P on the node interval of planes z1 (even) and z1 + 1, their
    // coordinates and the loads of their corners and of R, into registers that
    // are first used one step later
    auto a_issue = [&](int z1, bool first) {
        const int K1 = z1 >> 1;
        int qb[3] = {0, 0, 0};
        float fe[3] = {0.f, 0.f, 0.f}, fo[3] = {0.f, 0.f, 0.f};
        bool iv_ok = false;
        if (col_in) {
            float Ulo[3], Blo[3];
            if (first) {
                column_plane<HAS_DIR>(sm, K1, lkx, lky, wx, wy, t, Ulo, Blo);
            } else {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    Ulo[c] = Uhi[c];
                    Blo[c] = Bhi[c];
                }
            }
            column_plane<HAS_DIR>(sm, K1 + 1, lkx, lky, wx, wy, t, Uhi, Bhi);
            // y-hat = U_lo + lerp(B_lo, (U_hi - U_lo) + B_hi, wz) with wz = 1/4 (even z) or
            // 3/4 (odd z).  The sampling coordinate i + y-hat / h is kept as an integer
            // part plus a small fraction (see sample_coord); both depend only on the
            // interval and the parity of z, so they are formed here once.
            iv_ok = true;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float ih = g.ih[c];
                const float q0 = Ulo[c] * ih;
                const float d1 = (Uhi[c] - Ulo[c]) + Bhi[c];
                iv_ok = iv_ok && fabsf(q0) < 1.0e6f && fabsf(Blo[c] * ih) < 1.0e6f && fabsf(d1 * ih) < 1.0e6f;
                const float qi = floorf(q0);
                const float rem = fmaf(-qi, g.h[c], Ulo[c]);   // |rem| <~ h
                fe[c] = (rem + lerpf(Blo[c], d1, 0.25f)) * ih;
                fo[c] = (rem + lerpf(Blo[c], d1, 0.75f)) * ih;
                qb[c] = (int)qi;
            }
        }
        issue_node_plane(nc, sm, K1 + 2, g.n[2], node_plane);
        cp_async_commit();
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int zz = z1 + h;
            const bool zin = col_in && zz >= 0 && zz < mz;
#pragma unroll
            for (int k = 0; k < 8; k++)
                pc[h][k] = 0.f;
            int cc[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float f = h ? fo[c] : fe[c];
                const float fl = floorf(f);
                fr[h][c] = f - fl;
                cc[c] = qb[c] + (int)fl;
            }
            const int cx = cc[0] + x, cy = cc[1] + y, cz = cc[2] + zz;
            if (zin && iv_ok) {
                if ((unsigned)cx < (unsigned)(mx - 1) && (unsigned)cy < (unsigned)(my - 1) &&
                    (unsigned)cz < (unsigned)(mz - 1)) {   // all 8 corners inside
                    const IMG *p = Tim + (cx + mx * (cy + my * cz));
                    pc[h][0] = ldimg(p);
                    pc[h][1] = ldimg(p + 1);
                    pc[h][2] = ldimg(p + mx);
                    pc[h][3] = ldimg(p + mx + 1);
                    pc[h][4] = ldimg(p + sxy);
                    pc[h][5] = ldimg(p + sxy + 1);
                    pc[h][6] = ldimg(p + sxy + mx);
                    pc[h][7] = ldimg(p + sxy + mx + 1);
                } else {   // zero extension corner by corner
#pragma unroll
                    for (int k = 0; k < 8; k++)
                        pc[h][k] = ldimg_zero_ext(Tim, mx, my, mz, cx + (k & 1), cy + ((k >> 1) & 1), cz + (k >> 2));
                }
            }
            rnext[h] = zin ? ldimg(Rcol + sxy * zz) : 0.f;
        }
    };

    // prologue: node planes of the first interval, then the loads of planes z0 - 2, z0 - 1
    {
        const int K0 = (z0 - 2) >> 1;
        issue_node_plane(nc, sm, K0, g.n[2], node_plane);
        issue_node_plane(nc, sm, K0 + 1, g.n[2], node_plane);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        a_issue(z0 - 2, true);
        cp_async_wait_all();
        __syncthreads();
    }

    const int nsteps = a.tz / 2 + 5;
    for (int s = 0; s < nsteps; s++) {
        const int zA = z0 - 2 + 2 * s;
        // ---- A-finish: T~ and grad T on planes zA, zA + 1
        if (zA <= zend) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const float t000 = pc[h][0], t100 = pc[h][1], t010 = pc[h][2], t110 = pc[h][3];
                const float t001 = pc[h][4], t101 = pc[h][5], t011 = pc[h][6], t111 = pc[h][7];
                const float f0 = fr[h][0], f1 = fr[h][1], f2 = fr[h][2];
                const float a00 = lerpf(t000, t100, f0), a10 = lerpf(t010, t110, f0);
                const float a01 = lerpf(t001, t101, f0), a11 = lerpf(t011, t111, f0);
                const float b0 = lerpf(a00, a10, f1), b1 = lerpf(a01, a11, f1);
                const float val = lerpf(b0, b1, f2);
                const float dx0 = lerpf(t100 - t000, t110 - t010, f1), dx1 = lerpf(t101 - t001, t111 - t011, f1);
                const int slot = (zA + h) & 7;
                sm[OFF_T + slot * PLANE + tid] = val;
                sm[OFF_R + slot * PLANE + tid] = rnext[h];
                float *gq = sm + OFF_G + slot * 3 * PLANE + tid;
                gq[0] = lerpf(dx0, dx1, f2) * g.ih[0];
                gq[PLANE] = lerpf(a10 - a00, a11 - a01, f2) * g.ih[1];
                gq[2 * PLANE] = (b1 - b0) * g.ih[2];
            }
        }
        // ---- A-issue for planes zA + 2, zA + 3
        if (zA + 2 <= zend)
            a_issue(zA + 2, false);
        // ---- B: v on planes zA - 3, zA - 2 (rows 1 .. 14, lanes 1 .. 30)
        if (rowB && zA - 3 >= z0 - 1 && zA - 3 <= zend) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int zB = zA - 3 + h;
                float v[3] = {0.f, 0.f, 0.f};
                if (colB) {
                    if (intxy && zB >= 1 && zB <= mz - 2) {
                        const float *T0 = sm + OFF_T + (zB & 7) * PLANE + tid;
                        const float *R0 = sm + OFF_R + (zB & 7) * PLANE + tid;
                        float av[3], bv[3];
                        av[0] = (T0[1] - T0[-1]) * hx;
                        av[1] = (T0[BX] - T0[-BX]) * hy;
                        av[2] = (sm[OFF_T + ((zB + 1) & 7) * PLANE + tid] - sm[OFF_T + ((zB - 1) & 7) * PLANE + tid]) * hz;
                        bv[0] = (R0[1] - R0[-1]) * hx;
                        bv[1] = (R0[BX] - R0[-BX]) * hy;
                        bv[2] = (sm[OFF_R + ((zB + 1) & 7) * PLANE + tid] - sm[OFF_R + ((zB - 1) & 7) * PLANE + tid]) * hz;
                        const float psi = ngf_residual(av, bv, a.tau, a.rho, v);
                        if (colC && rowC && zB >= z0 && zB < zend)
                            psi_sum.add(psi);
                    }
                    float *vq = sm + OFF_V + (zB & 7) * 3 * PLANE + tid;
                    vq[0] = v[0];
                    vq[PLANE] = v[1];
                    vq[2 * PLANE] = v[2];
                }
            }
        }
        // ---- C: r on planes zA - 6, zA - 5 (rows 2 .. 13), x reduction into node columns
        if (rowC && zA - 6 >= z0 && zA - 5 < zend) {
            float *redb = sm + OFF_RED + (s & 1) * 2 * RED_PLANE + ty * NX * 3;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int zC = zA - 6 + h;
                float r[3] = {0.f, 0.f, 0.f};
                if (colC && col_in && zC < mz) {
                    const float *V0 = sm + OFF_V + (zC & 7) * 3 * PLANE + tid;
                    const float gs = (V0[-1] - V0[1]) * hx + (V0[PLANE - BX] - V0[PLANE + BX]) * hy +
                                     (sm[OFF_V + ((zC - 1) & 7) * 3 * PLANE + 2 * PLANE + tid] -
                                      sm[OFF_V + ((zC + 1) & 7) * 3 * PLANE + 2 * PLANE + tid]) * hz;
                    const float gj = half_hbar * gs;
                    const float *gq = sm + OFF_G + (zC & 7) * 3 * PLANE + tid;
                    r[0] = gj * gq[0];
                    r[1] = gj * gq[PLANE];
                    r[2] = gj * gq[2 * PLANE];
                }
                // node column j (0..14) gathers lanes 2j .. 2j+3 with weights 1/4, 3/4, 3/4, 1/4
                float *red = redb + h * RED_PLANE;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float r1 = __shfl_down_sync(0xffffffffu, r[c], 1);
                    const float r2 = __shfl_down_sync(0xffffffffu, r[c], 2);
                    const float r3 = __shfl_down_sync(0xffffffffu, r[c], 3);
                    // written nodes have tx = 2j <= 28, so lanes tx + 1 .. tx + 3 exist
                    if (!(tx & 1) && (tx >> 1) < NX)
                        red[(tx >> 1) * 3 + c] = 0.25f * (r[c] + r3) + 0.75f * (r1 + r2);
                }
            }
        }
        // ---- D: y reduction of planes zA - 8, zA - 7 (one node interval) and
        // accumulation of its two node planes along z
        if (dD && zA - 8 >= z0 && zA - 7 < zend) {
            const int lz = zA - 8 - z0;                   // even
            const float *red = sm + OFF_RED + ((s - 1) & 1) * 2 * RED_PLANE + dofs;
            const float v0 = 0.25f * red[0] + 0.75f * red[NX * 3] + 0.75f * red[2 * NX * 3] + 0.25f * red[3 * NX * 3];
            red += RED_PLANE;
            const float v1 = 0.25f * red[0] + 0.75f * red[NX * 3] + 0.75f * red[2 * NX * 3] + 0.25f * red[3 * NX * 3];
            // even plane: 3/4 to the lower node plane, 1/4 to the upper; odd plane: the reverse
            part_tile[(size_t)(lz >> 1) * NE + tid] = acc_lo + (0.75f * v0 + 0.25f * v1);
            acc_lo = 0.25f * v0 + 0.75f * v1;
            if (lz == a.tz - 2)
                part_tile[(size_t)(a.tz >> 1) * NE + tid] = acc_lo;
        }
        cp_async_wait_all();
        __syncthreads();
    }
    double ssum = block_sum_to_f64(psi_sum.s, reinterpret_cast<double *>(sm + OFF_RED));
    if (tid == 0)
        a.partials[tile_lin] = ssum;
}

template <bool HAS_DIR, typename IMG = float>
__global__ void __launch_bounds__(BX * BY, 1) k_ngf_fused(FusedArgs a)
{
    extern __shared__ float sm[];
    fused_tile<HAS_DIR, IMG>(a, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

// Batched fused pass: a persistent grid walks the tiles of all pairs.  Mode 0
// evaluates at u; mode 1 at the trial point, for the pairs still searching.
template <bool HAS_DIR, typename IMG>
__global__ void __launch_bounds__(BX * BY, 1) k_ngf_fused_batch(const PairLevel *__restrict__ pl,
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
        const int local = item - __ldg(tile_off + p);
        const int tx = local % a.ntx, rest = local / a.ntx;
        fused_tile<HAS_DIR, IMG>(a, tx, rest % a.nty, rest / a.nty, sm);
        __syncthreads();   // the next tile reuses the shared rings
    }
}

// grad J at node k = sum of the tile partials that contain k (P^T r) plus
// alpha hbar_y L^T w (curvature), one thread per node, 3 components.
__device__ __forceinline__ void gather_grad_body(const LevelGeom &g, const float *__restrict__ part, int tz, int ntx,
                                                 int nty, int ntz, const float *__restrict__ w, float alpha_hy,
                                                 float *__restrict__ grad, int bx, int by, int bz)
{
    int kx = bx * blockDim.x + threadIdx.x;
    int ky = by * blockDim.y + threadIdx.y;
    int kz = bz;
    if (kx >= g.n[0] || ky >= g.n[1])
        return;   // (only this function: a caller's barrier after it is still reached)
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

__global__ void __launch_bounds__(256) k_gather_grad(LevelGeom g, const float *__restrict__ part, int tz, int ntx,
                                                     int nty, int ntz, const float *__restrict__ w, float alpha_hy,
                                                     float *__restrict__ grad)
{
    gather_grad_body(g, part, tz, ntx, nty, ntz, w, alpha_hy, grad, blockIdx.x, blockIdx.y, blockIdx.z);
}

// The end of an evaluation after the gather: the block that completes the
// launch reduces the D and S block partials into scal = [J, D, S] (the fixed
// order of finalize_body) and, for phase >= 0, takes that L-BFGS control phase
// (the Armijo decision of a trial point) in the same block.
struct FinArgs {
    const double *pD, *pS;  // block partials of D (fused tiles) and S (curvature blocks)
    int nD, nS;
    double hbar_half, alpha, hy_half;
    double *scal;
    unsigned *cnt;          // arrival counter, zero between launches
    int phase;              // -1: no control phase
    LbfgsState *st;
    unsigned long long h_ls;
};

__global__ void __launch_bounds__(256) k_gather_fin(LevelGeom g, const float *__restrict__ part, int tz, int ntx,
                                                    int nty, int ntz, const float *__restrict__ w, float alpha_hy,
                                                    float *__restrict__ grad, FinArgs f)
{
    gather_grad_body(g, part, tz, ntx, nty, ntz, w, alpha_hy, grad, blockIdx.x, blockIdx.y, blockIdx.z);
    __shared__ int s_last;
    __syncthreads();
    if (linear_tid() == 0)
        s_last = atomicAdd(f.cnt, 1u) == gridDim.x * gridDim.y * gridDim.z - 1u;
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    finalize_body(f.pD, f.nD, f.pS, f.nS, f.hbar_half, f.alpha, f.hy_half, f.scal);
    if (linear_tid() == 0)
        *f.cnt = 0;
    if (f.phase >= 0) {
        __syncthreads();
        lb_control_body(f.phase, f.st, nullptr, 0, f.scal, f.h_ls, 0ULL, 0ULL);
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

// z segment lengths the autotuner tries (even: a segment covers whole node intervals)
constexpr int TZ_CAND[] = {2, 4, 8, 16, 32, 64, 128};

// Default z segment length when the level was not tuned: the longest of 8 ..
// 128 that still gives >= 2 CTAs per SM (each segment pays 7 pipeline-fill steps).
static int fused_tz_default(const Level &L, int num_sms)
{
    long long cols = (long long)((L.m[0] + OX - 1) / OX) * ((L.m[1] + OY - 1) / OY);
    int tz = 128;
    while (tz > 8 && cols * ((L.m[2] + tz - 1) / tz) < 2LL * num_sms)
        tz /= 2;
    return tz;
}

int fused_tz(const Level &L, int num_sms) { return L.tz > 0 ? L.tz : fused_tz_default(L, num_sms); }

// Throughput rule: the z segment length with the fewest z steps in total,
// ntz * (tz / 2 + 5) (ties: the longer one).  The right choice when other work
// keeps every SM busy (a batch of pairs); a single pair alone wants short
// segments that fill the GPU, which the autotuner finds.
int fused_tz_throughput(const Level &L)
{
    int best = 0;
    long long best_steps = 0;
    for (int tz : TZ_CAND) {
        const long long steps = (long long)((L.m[2] + tz - 1) / tz) * (tz / 2 + 5);
        if (best == 0 || steps <= best_steps) {
            best = tz;
            best_steps = steps;
        }
    }
    return best;
}

bool fused_tz_valid(int tz)
{
    for (int t : TZ_CAND)
        if (t == tz)
            return true;
    return false;
}

void fused_grid(const Level &L, int tz, int &ntx, int &nty, int &ntz)
{
    ntx = (L.m[0] + OX - 1) / OX;
    nty = (L.m[1] + OY - 1) / OY;
    ntz = (L.m[2] + tz - 1) / tz;
}

// tile-partial floats of the level: the largest over every z segment length
// the autotuner may pick
size_t fused_part_floats(const Level &L, int num_sms)
{
    (void)num_sms;
    size_t best = 0;
    for (int tz : TZ_CAND) {
        int ntx, nty, ntz;
        fused_grid(L, tz, ntx, nty, ntz);
        size_t p = (size_t)ntx * nty * ntz * (tz / 2 + 1) * NE;
        if (p > best)
            best = p;
    }
    return best;
}

cudaError_t launch_ngf_fused(reg_ctx *c, int level, const float *ub, const float *dir, const double *t_dev,
                             float *grad, double *partials, int *n_partials, cudaStream_t s)
{
    (void)grad;
    const Level &L = c->L[level];
    FusedArgs a;
    a.g = L.geom();
    const bool bf16 = c->cfg.image_dtype == 1 && L.Tb && L.Rb;
    a.T = bf16 ? L.Tb : static_cast<const void *>(L.T);
    a.R = bf16 ? L.Rb : static_cast<const void *>(L.R);
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
    // the shared rings exceed the 48 KB default; the limit is set once per device
    static bool attr_set[64] = {};
    const int dev = c->device >= 0 && c->device < 64 ? c->device : 0;
    if (!attr_set[dev]) {
        const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaError_t e = cudaFuncSetAttribute(k_ngf_fused<true, float>, at, (int)SMEM_BYTES);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_ngf_fused<false, float>, at, (int)SMEM_BYTES);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_ngf_fused<true, __nv_bfloat16>, at, (int)SMEM_BYTES);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_ngf_fused<false, __nv_bfloat16>, at, (int)SMEM_BYTES);
        if (e != cudaSuccess)
            return e;
        attr_set[dev] = true;
    }
    if (bf16) {
        if (dir)
            k_ngf_fused<true, __nv_bfloat16><<<grd, blk, SMEM_BYTES, s>>>(a);
        else
            k_ngf_fused<false, __nv_bfloat16><<<grd, blk, SMEM_BYTES, s>>>(a);
    } else {
        if (dir)
            k_ngf_fused<true, float><<<grd, blk, SMEM_BYTES, s>>>(a);
        else
            k_ngf_fused<false, float><<<grd, blk, SMEM_BYTES, s>>>(a);
    }
    *n_partials = a.ntx * a.nty * a.ntz;
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_gather_fin(reg_ctx *c, int level, const float *w, float alpha_hy, float *grad, int nD,
                              const double *pS, int nS, double *scal, int phase, cudaStream_t s)
{
    const Level &L = c->L[level];
    int tz = fused_tz(L, c->num_sms), ntx, nty, ntz;
    fused_grid(L, tz, ntx, nty, ntz);
    dim3 blk(32, 8, 1);
    dim3 gn((L.n[0] + 31) / 32, (L.n[1] + 7) / 8, L.n[2]);
    FinArgs f;
    f.pD = c->es.partials;
    f.nD = nD;
    f.pS = pS;
    f.nS = nS;
    f.hbar_half = 0.5 * L.h[0] * L.h[1] * L.h[2];
    f.alpha = c->cfg.alpha;
    f.hy_half = 0.5 * L.H[0] * L.H[1] * L.H[2];
    f.scal = scal;
    f.cnt = c->es.fin_cnt;
    f.phase = phase;
    f.st = c->lb.st;
    f.h_ls = phase >= 0 ? lbfgs_graph_handle_ls() : 0ULL;
    k_gather_fin<<<gn, blk, 0, s>>>(L.geom(), c->es.part, tz, ntx, nty, ntz, w, alpha_hy, grad, f);
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

// ---------------------------------------------------------------------------
// Autotuner of the z segment length (the tile depth of the fused pass).  For
// every candidate the pass runs on the level's own images at u = u_zero (one
// warm launch, then the median of three CUDA-event timings); the fastest wins.
// Short segments start more CTAs (small levels fill the GPU) but pay the 7
// pipeline-fill steps and the shared node planes more often, so the best
// depth depends on the level and the GPU.  Choices are cached per (image
// dims, SM count, image type, device) for the life of the process: handles of
// the same geometry tune once and pick the same tiling.
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::array<int, 6>, int> g_tune;
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
            L.tz = it->second;
            return cudaSuccess;
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    int best = 0;
    float best_ms = 0.f;
    for (int tz : TZ_CAND) {
        if (e != cudaSuccess)
            break;
        if (tz > 2 && tz / 2 >= L.m[2])   // the previous candidate already spans the whole depth
            break;
        L.tz = tz;
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
        if (best == 0 || med < best_ms) {
            best = tz;
            best_ms = med;
        }
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        L.tz = 0;
        return e;
    }
    L.tz = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Explicit-buffer launches of the fused pass and its gather, for callers that
// own every buffer themselves (the allocation-free entry point).  Geometry
// comes in as a LevelGeom of a ratio-2 grid; no per-dimension tables are used.
// ---------------------------------------------------------------------------
static int fused_tz_dims(const int m[3], int num_sms)
{
    long long cols = (long long)((m[0] + OX - 1) / OX) * ((m[1] + OY - 1) / OY);
    int tz = 64;
    while (tz > 8 && cols * ((m[2] + tz - 1) / tz) < 2LL * num_sms)
        tz /= 2;
    return tz;
}

void fused_layout_dims(const int m[3], int num_sms, int *tz, int *tiles, size_t *part_floats)
{
    const int z = fused_tz_dims(m, num_sms);
    const int nt = ((m[0] + OX - 1) / OX) * ((m[1] + OY - 1) / OY) * ((m[2] + z - 1) / z);
    *tz = z;
    *tiles = nt;
    *part_floats = (size_t)nt * (z / 2 + 1) * NE;
}

cudaError_t fused_set_smem_limit()
{
    cudaError_t e = cudaFuncSetAttribute(k_ngf_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ngf_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    return e;
}

cudaError_t launch_ngf_fused_raw(const LevelGeom &g, const float *T, const float *R, const float *u, float tau,
                                 float rho, int num_sms, float *part, double *partials, cudaStream_t s)
{
    FusedArgs a;
    a.g = g;
    a.T = T;
    a.R = R;
    a.ub = u;
    a.dir = nullptr;
    a.t_dev = nullptr;
    a.tau = tau;
    a.rho = rho;
    a.tz = fused_tz_dims(g.m, num_sms);
    a.ntx = (g.m[0] + OX - 1) / OX;
    a.nty = (g.m[1] + OY - 1) / OY;
    a.ntz = (g.m[2] + a.tz - 1) / a.tz;
    a.part = part;
    a.partials = partials;
    dim3 blk(BX, BY, 1), grd(a.ntx, a.nty, a.ntz);
    k_ngf_fused<false><<<grd, blk, SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gather_grad_raw(const LevelGeom &g, const float *part, int num_sms, const float *w,
                                   float alpha_hy, float *grad, cudaStream_t s)
{
    const int tz = fused_tz_dims(g.m, num_sms);
    const int ntx = (g.m[0] + OX - 1) / OX, nty = (g.m[1] + OY - 1) / OY, ntz = (g.m[2] + tz - 1) / tz;
    dim3 blk(32, 8, 1);
    dim3 gn((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, g.n[2]);
    k_gather_grad<<<gn, blk, 0, s>>>(g, part, tz, ntx, nty, ntz, w, alpha_hy, grad);
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
        const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaError_t e = cudaFuncSetAttribute(k_ngf_fused_batch<true, float>, at, (int)SMEM_BYTES);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_ngf_fused_batch<false, float>, at, (int)SMEM_BYTES);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_ngf_fused_batch<true, __nv_bfloat16>, at, (int)SMEM_BYTES);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_ngf_fused_batch<false, __nv_bfloat16>, at, (int)SMEM_BYTES);
        if (e != cudaSuccess)
            return e;
        g_batch_attr_set[dev] = true;
    }
    dim3 blk(BX, BY, 1);
    if (bf16) {
        if (mode)
            k_ngf_fused_batch<true, __nv_bfloat16><<<grid, blk, SMEM_BYTES, s>>>(pl, tile_off, npairs, total);
        else
            k_ngf_fused_batch<false, __nv_bfloat16><<<grid, blk, SMEM_BYTES, s>>>(pl, tile_off, npairs, total);
    } else {
        if (mode)
            k_ngf_fused_batch<true, float><<<grid, blk, SMEM_BYTES, s>>>(pl, tile_off, npairs, total);
        else
            k_ngf_fused_batch<false, float><<<grid, blk, SMEM_BYTES, s>>>(pl, tile_off, npairs, total);
    }
    return cudaGetLastError();
}

namespace {

__global__ void __launch_bounds__(256) k_gather_batch(const PairLevel *__restrict__ pl, const int *__restrict__ off,
                                                      int npairs, int total, int mode)
{
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int p = find_pair(off, npairs, item);
        const PairLevel &P = pl[p];
        if (mode == 1 && !(P.st->active && P.st->ls_continue))
            continue;
        const int lin = item - __ldg(off + p);
        const int bx = lin % P.ncx, r = lin / P.ncx;
        const FusedArgs &a = P.fa_init;
        gather_grad_body(P.geom, a.part, a.tz, a.ntx, a.nty, a.ntz, P.w, P.alpha_hy, mode ? P.gt : P.g, bx,
                         r % P.ncy, r / P.ncy);
    }
}

}  // namespace

cudaError_t launch_gather_batch(const PairLevel *pl, const int *off, int npairs, int total, int mode, int grid,
                                cudaStream_t s)
{
    k_gather_batch<<<grid, dim3(32, 8, 1), 0, s>>>(pl, off, npairs, total, mode);
    return cudaGetLastError();
}

// tiling of a level of the fused pass, for the batch descriptors
void fused_tiling(const Level &L, int num_sms, int *tz, int *ntx, int *nty, int *ntz)
{
    *tz = fused_tz(L, num_sms);
    fused_grid(L, *tz, *ntx, *nty, *ntz);
}
