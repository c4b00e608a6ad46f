// Multi-pass objective evaluation: one kernel per step of Sec. 2.2
// "Evaluating the objective function", intermediates in HBM.  It is the
// plain-structured variant kept beside the fused pass (reg_config.eval_impl =
// 1), used to cross-check it and as the A/B baseline for its traffic.
//
//   k_mp_warp   : y-hat = P u (Eq. 1), T(x + y-hat) and the interpolant gradient
//   k_mp_resid  : NGF residual on interior voxels (Eq. 2), v = d psi / d grad T
//   k_mp_adjoint: g = adjoint central difference of v, r = g grad T (chain rule)
//   k_mp_pt     : grad D = P^T r as the node-centric gather of Eq. 3
//
// Two A/B variants of the last two steps measure what the gather form of
// Eq. 3 buys (Sec. 2.2 names both as slower designs it replaced):
//   eval_impl 2, k_mp_adjoint_atomic: r per voxel, scattered to its 8 nodes
//     with atomicAdd (summation order not fixed);
//   eval_impl 3, k_mp_adjoint_colour: ratio-2 grids only; a thread owns the
//     2 x 2 x 2 voxels of one node cell (voxels 2k, 2k+1 per dimension lie in
//     cell [k, k+1]) and writes the cell's 8 nodes without atomics; cells of
//     equal (k_x, k_y, k_z) parity never share a node, so 8 launches (one per
//     parity colour) cover the grid in a fixed order.
#include "internal.h"
#include "ngf_math.cuh"

namespace {

__global__ void __launch_bounds__(256) k_mp_warp(LevelGeom g, const float *__restrict__ T,
                                                 const float *__restrict__ ub, const float *__restrict__ dir,
                                                 const double *__restrict__ t_dev, float *__restrict__ Tw,
                                                 float *__restrict__ dT)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int z = blockIdx.z;
    if (x >= g.m[0] || y >= g.m[1])
        return;
    float t = dir ? (float)__ldg(t_dev) : 0.f;
    float val, gr[3];
    warp_voxel(g, T, ub, dir, t, x, y, z, val, gr);
    size_t i = x + (size_t)g.m[0] * (y + (size_t)g.m[1] * z);
    Tw[i] = val;
    dT[i] = gr[0];
    dT[g.nv + i] = gr[1];
    dT[2 * g.nv + i] = gr[2];
}

__global__ void __launch_bounds__(256) k_mp_resid(LevelGeom g, const float *__restrict__ Tw,
                                                  const float *__restrict__ R, float tau, float rho,
                                                  float *__restrict__ v, double *__restrict__ partials)
{
    __shared__ double sm[8];
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int z = blockIdx.z;
    bool in = x < g.m[0] && y < g.m[1];
    float psi = 0.f, vv[3] = {0.f, 0.f, 0.f};
    size_t i = in ? x + (size_t)g.m[0] * (y + (size_t)g.m[1] * z) : 0;
    if (in && x >= 1 && y >= 1 && z >= 1 && x <= g.m[0] - 2 && y <= g.m[1] - 2 && z <= g.m[2] - 2) {
        size_t st[3] = {1, (size_t)g.m[0], (size_t)g.m[0] * g.m[1]};
        float a[3], b[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            a[d] = (__ldg(Tw + i + st[d]) - __ldg(Tw + i - st[d])) * (0.5f * g.ih[d]);
            b[d] = (__ldg(R + i + st[d]) - __ldg(R + i - st[d])) * (0.5f * g.ih[d]);
        }
        psi = ngf_residual(a, b, tau, rho, vv);
    }
    if (in) {
        v[i] = vv[0];
        v[g.nv + i] = vv[1];
        v[2 * g.nv + i] = vv[2];
    }
    double s = block_sum_to_f64(psi, sm);
    if (linear_tid() == 0)
        partials[linear_bid()] = s;
}

__global__ void __launch_bounds__(256) k_mp_adjoint(LevelGeom g, const float *__restrict__ v,
                                                    const float *__restrict__ dT, float *__restrict__ r)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int z = blockIdx.z;
    if (x >= g.m[0] || y >= g.m[1])
        return;
    size_t i = x + (size_t)g.m[0] * (y + (size_t)g.m[1] * z);
    size_t st[3] = {1, (size_t)g.m[0], (size_t)g.m[0] * g.m[1]};
    int j[3] = {x, y, z};
    float s = 0.f;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float *vd = v + d * g.nv;
        float lo = j[d] > 0 ? __ldg(vd + i - st[d]) : 0.f;
        float hi = j[d] < g.m[d] - 1 ? __ldg(vd + i + st[d]) : 0.f;
        s = fmaf(lo - hi, 0.5f * g.ih[d], s);
    }
    float gj = 0.5f * g.hbar * s;
#pragma unroll
    for (int c = 0; c < 3; c++)
        r[c * g.nv + i] = gj * __ldg(dT + c * g.nv + i);
}

// Eq. 3: node k sums omega * r_i over Omega_1(k_x) x Omega_2(k_y) x Omega_3(k_z).
__global__ void __launch_bounds__(256) k_mp_pt(LevelGeom g, const float *__restrict__ r, float *__restrict__ out)
{
    int kx = blockIdx.x * blockDim.x + threadIdx.x;
    int ky = blockIdx.y * blockDim.y + threadIdx.y;
    int kz = blockIdx.z;
    if (kx >= g.n[0] || ky >= g.n[1])
        return;
    int fx = g.tfirst[0][kx], cx = g.tcnt[0][kx];
    int fy = g.tfirst[1][ky], cy = g.tcnt[1][ky];
    int fz = g.tfirst[2][kz], cz = g.tcnt[2][kz];
    const float *wx = g.tw[0] + (size_t)kx * g.tmaxw[0];
    const float *wy = g.tw[1] + (size_t)ky * g.tmaxw[1];
    const float *wz = g.tw[2] + (size_t)kz * g.tmaxw[2];
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int c = 0; c < cz; c++) {
        for (int b = 0; b < cy; b++) {
            float wzy = wz[c] * wy[b];
            size_t row = (size_t)fx + (size_t)g.m[0] * ((size_t)(fy + b) + (size_t)g.m[1] * (fz + c));
            for (int a = 0; a < cx; a++) {
                float w = wzy * wx[a];
                s0 = fmaf(w, __ldg(r + row + a), s0);
                s1 = fmaf(w, __ldg(r + g.nv + row + a), s1);
                s2 = fmaf(w, __ldg(r + 2 * g.nv + row + a), s2);
            }
        }
    }
    size_t k = kx + (size_t)g.n[0] * (ky + (size_t)g.n[1] * kz);
    out[k] = s0;
    out[g.nn + k] = s1;
    out[2 * g.nn + k] = s2;
}

// r at voxel (x, y, z): the adjoint central difference of v times grad T
__device__ __forceinline__ void mp_r(const LevelGeom &g, const float *__restrict__ v, const float *__restrict__ dT,
                                     int x, int y, int z, float r[3])
{
    size_t i = x + (size_t)g.m[0] * (y + (size_t)g.m[1] * z);
    size_t st[3] = {1, (size_t)g.m[0], (size_t)g.m[0] * g.m[1]};
    int j[3] = {x, y, z};
    float s = 0.f;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float *vd = v + d * g.nv;
        float lo = j[d] > 0 ? __ldg(vd + i - st[d]) : 0.f;
        float hi = j[d] < g.m[d] - 1 ? __ldg(vd + i + st[d]) : 0.f;
        s = fmaf(lo - hi, 0.5f * g.ih[d], s);
    }
    float gj = 0.5f * g.hbar * s;
#pragma unroll
    for (int c = 0; c < 3; c++)
        r[c] = gj * __ldg(dT + c * g.nv + i);
}

// A/B variant: r scattered to the 8 nodes of the voxel's cell by atomicAdd
// (P's weights from the per-dimension tables: node k0 weight 1 - w1, k0 + 1 weight w1).
__global__ void __launch_bounds__(256) k_mp_adjoint_atomic(LevelGeom g, const float *__restrict__ v,
                                                           const float *__restrict__ dT, float *__restrict__ out)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int z = blockIdx.z;
    if (x >= g.m[0] || y >= g.m[1])
        return;
    float r[3];
    mp_r(g, v, dT, x, y, z, r);
    const int kx = g.pk0[0][x], ky = g.pk0[1][y], kz = g.pk0[2][z];
    const float wx = g.pw1[0][x], wy = g.pw1[1][y], wz = g.pw1[2][z];
#pragma unroll
    for (int n = 0; n < 8; n++) {
        const int a = n & 1, b = (n >> 1) & 1, cz = n >> 2;
        const float w = (a ? wx : 1.f - wx) * (b ? wy : 1.f - wy) * (cz ? wz : 1.f - wz);
        const size_t k = (kx + a) + (size_t)g.n[0] * ((ky + b) + (size_t)g.n[1] * (kz + cz));
#pragma unroll
        for (int c = 0; c < 3; c++)
            atomicAdd(out + c * g.nn + k, w * r[c]);
    }
}

// A/B variant: one thread per node cell of one parity colour, no atomics
// (ratio-2 grids: voxels 2k, 2k+1 in cell k, weights 3/4, 1/4 of nodes k, k+1
// for voxel 2k and 1/4, 3/4 for voxel 2k+1).
__global__ void __launch_bounds__(256) k_mp_adjoint_colour(LevelGeom g, const float *__restrict__ v,
                                                           const float *__restrict__ dT, float *__restrict__ out,
                                                           int colour)
{
    const int cx = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + (colour & 1);
    const int cy = 2 * (blockIdx.y * blockDim.y + threadIdx.y) + ((colour >> 1) & 1);
    const int cz = 2 * blockIdx.z + (colour >> 2);
    if (cx >= g.n[0] - 1 || cy >= g.n[1] - 1 || cz >= g.n[2] - 1)
        return;
    float acc[8][3];
#pragma unroll
    for (int n = 0; n < 8; n++)
#pragma unroll
        for (int c = 0; c < 3; c++)
            acc[n][c] = 0.f;
#pragma unroll
    for (int q = 0; q < 8; q++) {   // the cell's voxels
        const int qx = q & 1, qy = (q >> 1) & 1, qz = q >> 2;
        float r[3];
        mp_r(g, v, dT, 2 * cx + qx, 2 * cy + qy, 2 * cz + qz, r);
        const float wx = qx ? 0.75f : 0.25f, wy = qy ? 0.75f : 0.25f, wz = qz ? 0.75f : 0.25f;
#pragma unroll
        for (int n = 0; n < 8; n++) {
            const int a = n & 1, b = (n >> 1) & 1, e = n >> 2;
            const float w = (a ? wx : 1.f - wx) * (b ? wy : 1.f - wy) * (e ? wz : 1.f - wz);
#pragma unroll
            for (int c = 0; c < 3; c++)
                acc[n][c] = fmaf(w, r[c], acc[n][c]);
        }
    }
#pragma unroll
    for (int n = 0; n < 8; n++) {
        const size_t k = (cx + (n & 1)) + (size_t)g.n[0] * ((cy + ((n >> 1) & 1)) + (size_t)g.n[1] * (cz + (n >> 2)));
#pragma unroll
        for (int c = 0; c < 3; c++)
            out[c * g.nn + k] += acc[n][c];
    }
}

}  // namespace

// Multi-pass D and grad D; D block partials go to partials[0 .. returned count).
cudaError_t launch_ngf_multipass(reg_ctx *c, int level, const float *ub, const float *dir, const double *t_dev,
                                 float *grad, double *partials, int *n_partials, cudaStream_t s)
{
    const Level &L = c->L[level];
    LevelGeom g = L.geom();
    dim3 blk(32, 8, 1);
    dim3 gv((L.m[0] + 31) / 32, (L.m[1] + 7) / 8, L.m[2]);
    dim3 gn((L.n[0] + 31) / 32, (L.n[1] + 7) / 8, L.n[2]);
    k_mp_warp<<<gv, blk, 0, s>>>(g, L.T, ub, dir, t_dev, c->es.Tw, c->es.dT);
    k_mp_resid<<<gv, blk, 0, s>>>(g, c->es.Tw, L.R, (float)c->cfg.tau, (float)c->cfg.rho, c->es.v, partials);
    *n_partials = (int)(gv.x * gv.y * gv.z);
    const int pt = mp_pt_variant(c, level);
    if (pt == 0) {   // node-centric gather (Eq. 3)
        k_mp_adjoint<<<gv, blk, 0, s>>>(g, c->es.v, c->es.dT, c->es.r);
        k_mp_pt<<<gn, blk, 0, s>>>(g, c->es.r, grad);
        c->launches += 4;
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * 3 * L.nn, s);
    if (e != cudaSuccess)
        return e;
    if (pt == 1) {   // atomic scatter
        k_mp_adjoint_atomic<<<gv, blk, 0, s>>>(g, c->es.v, c->es.dT, grad);
        c->launches += 3;
        return cudaGetLastError();
    }
    // 8-colour scatter over the node cells
    const int cells[3] = {L.n[0] - 1, L.n[1] - 1, L.n[2] - 1};
    dim3 gc(((cells[0] + 1) / 2 + 31) / 32, ((cells[1] + 1) / 2 + 7) / 8, (cells[2] + 1) / 2);
    for (int colour = 0; colour < 8; colour++)
        k_mp_adjoint_colour<<<gc, blk, 0, s>>>(g, c->es.v, c->es.dT, grad, colour);
    c->launches += 10;
    return cudaGetLastError();
}
