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

// Sampling coordinate of one voxel along one axis, t = i + yhat / h (voxel
// units, so that T's sample j sits at t = j), returned as an integer cell
// c = floor(t) and a fraction f = t - c in [0, 1).
//
// yhat = u0 + delta, where u0 is the displacement at the voxel's first node
// (an FP32 input value) and delta the trilinear interpolation of the node
// differences u_k - u0 (small for smooth fields).  Splitting off the integer
// part before adding delta keeps the absolute error of t near 1e-7 instead of
// the ~1e-5 that a float i + yhat / h has at i ~ 256: the interpolant's
// gradient jumps at cell faces, so a coordinate rounded across a face changes
// that voxel's gradient contribution completely.
// ok = false when the coordinate is not finite or absurdly far away.
__device__ __forceinline__ void sample_coord(int i, float u0, float delta, float h, float ih, int &c, float &f,
                                             bool &ok)
{
    float q0 = u0 * ih;
    ok = fabsf(q0) < 1.0e6f && fabsf(delta * ih) < 1.0e6f;   // also false for NaN
    float qi = floorf(q0);
    float rem = fmaf(-qi, h, u0);          // u0 - qi h with one rounding, |rem| <~ h
    float fr = (rem + delta) * ih;
    float ff = floorf(fr);
    f = fr - ff;
    c = ok ? i + (int)qi + (int)ff : 0;
}

// Grid conversion P at one voxel (Sec. 2.1 Eq. 1, Sec. 2.2): trilinear in the
// 8 surrounding nodes with the per-dimension weights; per component the value
// at the first node (u0) and the interpolated differences to it (delta).
__device__ __forceinline__ void grid_convert_point(const LevelGeom &g, const float *__restrict__ ub,
                                                   const float *__restrict__ dir, float t, int x, int y, int z,
                                                   float u0[3], float delta[3])
{
    int kx = __ldg(g.pk0[0] + x), ky = __ldg(g.pk0[1] + y), kz = __ldg(g.pk0[2] + z);
    float wx = __ldg(g.pw1[0] + x), wy = __ldg(g.pw1[1] + y), wz = __ldg(g.pw1[2] + z);
    size_t sy = (size_t)g.n[0], sz = (size_t)g.n[0] * g.n[1];
    size_t b = kx + ky * sy + kz * sz;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float *u = ub + c * g.nn;
        const float *d = dir ? dir + c * g.nn : nullptr;
        float a = node_value(u, d, t, b);
        float d100 = node_value(u, d, t, b + 1) - a;
        float d010 = node_value(u, d, t, b + sy) - a, d110 = node_value(u, d, t, b + sy + 1) - a;
        float d001 = node_value(u, d, t, b + sz) - a, d101 = node_value(u, d, t, b + sz + 1) - a;
        float d011 = node_value(u, d, t, b + sz + sy) - a, d111 = node_value(u, d, t, b + sz + sy + 1) - a;
        float a0 = wx * d100;
        float a1 = lerpf(d010, d110, wx);
        float a2 = lerpf(d001, d101, wx);
        float a3 = lerpf(d011, d111, wx);
        u0[c] = a;
        delta[c] = lerpf(lerpf(a0, a1, wy), lerpf(a2, a3, wy), wz);
    }
}

__device__ __forceinline__ float load_zero_ext(const float *__restrict__ T, int mx, int my, int mz, int x, int y,
                                               int z)
{
    bool in = (unsigned)x < (unsigned)mx && (unsigned)y < (unsigned)my && (unsigned)z < (unsigned)mz;
    return in ? __ldg(T + (x + mx * (y + my * z))) : 0.f;
}

// Trilinear interpolation of T at cell c + fraction f (voxel units, sample j at
// t = j) with zero extension, and the gradient of the interpolant in that cell
// (per mm, through ih = 1 / h).  Index arithmetic is 32-bit (volumes below
// 2^31 voxels).  Cells whose 8 corners are all inside take a path with one
// bounds test; cells on the border load each corner with its own test.
__device__ __forceinline__ void interp_value_grad(const float *__restrict__ T, int mx, int my, int mz, const int c[3],
                                                  const float f[3], bool ok, const float ih[3], float &val,
                                                  float gr[3])
{
    const int cx = c[0], cy = c[1], cz = c[2];
    const int sxy = mx * my;
    float t000, t100, t010, t110, t001, t101, t011, t111;
    if (ok && (unsigned)cx < (unsigned)(mx - 1) && (unsigned)cy < (unsigned)(my - 1) &&
        (unsigned)cz < (unsigned)(mz - 1)) {
        const float *p = T + (cx + mx * (cy + my * cz));
        t000 = __ldg(p);
        t100 = __ldg(p + 1);
        t010 = __ldg(p + mx);
        t110 = __ldg(p + mx + 1);
        t001 = __ldg(p + sxy);
        t101 = __ldg(p + sxy + 1);
        t011 = __ldg(p + sxy + mx);
        t111 = __ldg(p + sxy + mx + 1);
    } else if (ok && cx >= -1 && cx <= mx - 1 && cy >= -1 && cy <= my - 1 && cz >= -1 && cz <= mz - 1) {
        t000 = load_zero_ext(T, mx, my, mz, cx, cy, cz);
        t100 = load_zero_ext(T, mx, my, mz, cx + 1, cy, cz);
        t010 = load_zero_ext(T, mx, my, mz, cx, cy + 1, cz);
        t110 = load_zero_ext(T, mx, my, mz, cx + 1, cy + 1, cz);
        t001 = load_zero_ext(T, mx, my, mz, cx, cy, cz + 1);
        t101 = load_zero_ext(T, mx, my, mz, cx + 1, cy, cz + 1);
        t011 = load_zero_ext(T, mx, my, mz, cx, cy + 1, cz + 1);
        t111 = load_zero_ext(T, mx, my, mz, cx + 1, cy + 1, cz + 1);
    } else {   // every corner outside (or a non-finite coordinate)
        val = 0.f;
        gr[0] = gr[1] = gr[2] = 0.f;
        return;
    }
    const float tx = f[0], ty = f[1], tz = f[2];
    float a00 = lerpf(t000, t100, tx), a10 = lerpf(t010, t110, tx);
    float a01 = lerpf(t001, t101, tx), a11 = lerpf(t011, t111, tx);
    float b0 = lerpf(a00, a10, ty), b1 = lerpf(a01, a11, ty);
    val = lerpf(b0, b1, tz);
    float dx0 = lerpf(t100 - t000, t110 - t010, ty), dx1 = lerpf(t101 - t001, t111 - t011, ty);
    gr[0] = lerpf(dx0, dx1, tz) * ih[0];
    gr[1] = lerpf(a10 - a00, a11 - a01, tz) * ih[1];
    gr[2] = (b1 - b0) * ih[2];
}

// Deformed-template value and interpolant gradient at voxel (x, y, z):
// y-hat = P u, then T(x + y-hat) (Eq. 1).
__device__ __forceinline__ void warp_voxel(const LevelGeom &g, const float *__restrict__ T,
                                           const float *__restrict__ ub, const float *__restrict__ dir, float t,
                                           int x, int y, int z, float &val, float gr[3])
{
    float u0[3], dl[3];
    grid_convert_point(g, ub, dir, t, x, y, z, u0, dl);
    int c[3];
    float f[3];
    bool ok0, ok1, ok2;
    sample_coord(x, u0[0], dl[0], g.h[0], g.ih[0], c[0], f[0], ok0);
    sample_coord(y, u0[1], dl[1], g.h[1], g.ih[1], c[1], f[1], ok1);
    sample_coord(z, u0[2], dl[2], g.h[2], g.ih[2], c[2], f[2], ok2);
    interp_value_grad(T, g.m[0], g.m[1], g.m[2], c, f, ok0 && ok1 && ok2, g.ih, val, gr);
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
    float psi = __fdividef(num, den);   // approximate division: ~2 ulp
    float rs = rsqrtf(den);            // 1 / (||a||_tau ||b||_rho)
    float c = (ab + tau * rho) * rs;
    float k1 = -2.f * c * rs;          // v = -2c (b / (na nb) - c a / na^2)
    float k2 = __fdividef(2.f * c * c, na2);
    v[0] = fmaf(k1, b[0], k2 * a[0]);
    v[1] = fmaf(k1, b[1], k2 * a[1]);
    v[2] = fmaf(k1, b[2], k2 * a[2]);
    return psi;
}
