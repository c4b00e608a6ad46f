// Per-point arithmetic of the objective, shared by the fused and the
// multi-pass evaluation kernels.
#pragma once

#include "common.cuh"

// Node value of the displacement at the current trial point u_b + t * dir
// (dir == nullptr: u_b).  The same fmaf is used when the accepted step is
// written back, so the accepted iterate equals the evaluated one bit for bit.
__device__ __forceinline__ float node_value(const float *__restrict__ ub, const float *__restrict__ dir, float t,
                                            size_t k)
{
    float v = __ldg(ub + k);
    if (dir)
        v = fmaf(t, __ldg(dir + k), v);
    return v;
}

// Grid conversion P at one voxel (Sec. 2.1 Eq. 1, Sec. 2.2): trilinear in the
// 8 surrounding nodes, weights from the per-dimension tables.
__device__ __forceinline__ void grid_convert_point(const LevelGeom &g, const float *__restrict__ ub,
                                                   const float *__restrict__ dir, float t, int x, int y, int z,
                                                   float yh[3])
{
    int kx = __ldg(g.pk0[0] + x), ky = __ldg(g.pk0[1] + y), kz = __ldg(g.pk0[2] + z);
    float wx = __ldg(g.pw1[0] + x), wy = __ldg(g.pw1[1] + y), wz = __ldg(g.pw1[2] + z);
    size_t sy = (size_t)g.n[0], sz = (size_t)g.n[0] * g.n[1];
    size_t b = kx + ky * sy + kz * sz;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float *u = ub + c * g.nn;
        const float *d = dir ? dir + c * g.nn : nullptr;
        float a0 = lerpf(node_value(u, d, t, b), node_value(u, d, t, b + 1), wx);
        float a1 = lerpf(node_value(u, d, t, b + sy), node_value(u, d, t, b + sy + 1), wx);
        float a2 = lerpf(node_value(u, d, t, b + sz), node_value(u, d, t, b + sz + 1), wx);
        float a3 = lerpf(node_value(u, d, t, b + sz + sy), node_value(u, d, t, b + sz + sy + 1), wx);
        yh[c] = lerpf(lerpf(a0, a1, wy), lerpf(a2, a3, wy), wz);
    }
}

__device__ __forceinline__ float load_zero_ext(const float *__restrict__ T, int mx, int my, int mz, int x, int y,
                                               int z)
{
    bool in = (unsigned)x < (unsigned)mx && (unsigned)y < (unsigned)my && (unsigned)z < (unsigned)mz;
    return in ? __ldg(T + x + (size_t)mx * (y + (size_t)my * z)) : 0.f;
}

// Trilinear interpolation of T at voxel-index coordinates s (s_d = p_d / h_d - 1/2)
// with zero extension, and the gradient of the interpolant in the cell
// floor(s) (per mm, through ih = 1 / h).
__device__ __forceinline__ void interp_value_grad(const float *__restrict__ T, int mx, int my, int mz,
                                                  const float s[3], const float ih[3], float &val, float gr[3])
{
    // outside (-1 <= s_d < m_d) every corner is outside; also catches NaN
    if (!(s[0] >= -1.f && s[0] < (float)mx && s[1] >= -1.f && s[1] < (float)my && s[2] >= -1.f &&
          s[2] < (float)mz)) {
        val = 0.f;
        gr[0] = gr[1] = gr[2] = 0.f;
        return;
    }
    float fx = floorf(s[0]), fy = floorf(s[1]), fz = floorf(s[2]);
    int cx = (int)fx, cy = (int)fy, cz = (int)fz;
    float tx = s[0] - fx, ty = s[1] - fy, tz = s[2] - fz;
    float t000 = load_zero_ext(T, mx, my, mz, cx, cy, cz);
    float t100 = load_zero_ext(T, mx, my, mz, cx + 1, cy, cz);
    float t010 = load_zero_ext(T, mx, my, mz, cx, cy + 1, cz);
    float t110 = load_zero_ext(T, mx, my, mz, cx + 1, cy + 1, cz);
    float t001 = load_zero_ext(T, mx, my, mz, cx, cy, cz + 1);
    float t101 = load_zero_ext(T, mx, my, mz, cx + 1, cy, cz + 1);
    float t011 = load_zero_ext(T, mx, my, mz, cx, cy + 1, cz + 1);
    float t111 = load_zero_ext(T, mx, my, mz, cx + 1, cy + 1, cz + 1);
    float a00 = lerpf(t000, t100, tx), a10 = lerpf(t010, t110, tx);
    float a01 = lerpf(t001, t101, tx), a11 = lerpf(t011, t111, tx);
    float b0 = lerpf(a00, a10, ty), b1 = lerpf(a01, a11, ty);
    val = lerpf(b0, b1, tz);
    float dx0 = lerpf(t100 - t000, t110 - t010, ty), dx1 = lerpf(t101 - t001, t111 - t011, ty);
    gr[0] = lerpf(dx0, dx1, tz) * ih[0];
    gr[1] = lerpf(a10 - a00, a11 - a01, tz) * ih[1];
    gr[2] = (b1 - b0) * ih[2];
}

// NGF residual of Eq. 2 at one interior voxel, a = grad T-tilde, b = grad R.
// Returns psi = 1 - c^2 and writes v = d psi / d a.  psi is evaluated through
// the exact identity
//   (|a|^2 + tau^2)(|b|^2 + rho^2) - (a.b + tau rho)^2 = |a x b|^2 + |tau b - rho a|^2,
// so no cancellation occurs when c is close to 1 (aligned or flat regions).
__device__ __forceinline__ float ngf_residual(const float a[3], const float b[3], float tau, float rho, float v[3])
{
    float aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    float bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    float ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    float na2 = aa + tau * tau, nb2 = bb + rho * rho;
    float cx = a[1] * b[2] - a[2] * b[1];
    float cy = a[2] * b[0] - a[0] * b[2];
    float cz = a[0] * b[1] - a[1] * b[0];
    float ex = tau * b[0] - rho * a[0], ey = tau * b[1] - rho * a[1], ez = tau * b[2] - rho * a[2];
    float num = cx * cx + cy * cy + cz * cz + ex * ex + ey * ey + ez * ez;
    float den = na2 * nb2;
    float psi = num / den;
    float rs = rsqrtf(den);            // 1 / (||a||_tau ||b||_rho)
    float c = (ab + tau * rho) * rs;
    float k1 = -2.f * c * rs;          // v = -2c (b / (na nb) - c a / na^2)
    float k2 = 2.f * c * c / na2;
    v[0] = fmaf(k1, b[0], k2 * a[0]);
    v[1] = fmaf(k1, b[1], k2 * a[1]);
    v[2] = fmaf(k1, b[2], k2 * a[2]);
    return psi;
}
