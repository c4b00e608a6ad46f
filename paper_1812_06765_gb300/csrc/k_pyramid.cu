// Pyramid generation and multilevel prolongation.
//
// Pyramid (Sec. 2.2 "Generating the multi-level pyramid"): each coarser level
// is the 2x2x2 mean of the finer one (an odd dimension replicates its last
// slab), spacing doubles.  The reference and template pyramids run on two
// streams.  Prolongation (Sec. 2.1, coarse-to-fine): nodal trilinear
// interpolation of the coarse displacement onto the finer nodes, with
// per-dimension (first node, weight) tables.
#include "internal.h"

namespace {

// One thread per output voxel; a warp covers 32 consecutive x of one row, so
// the two input rows it reads are contiguous 64-float spans.
__global__ void k_restrict(const float *__restrict__ src, int mx, int my, int mz, float *__restrict__ dst,
                           int ox, int oy, int oz)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int z = blockIdx.z;
    if (x >= ox || y >= oy)
        return;
    int x0 = 2 * x, x1 = min(2 * x + 1, mx - 1);
    int y0 = 2 * y, y1 = min(2 * y + 1, my - 1);
    int z0 = 2 * z, z1 = min(2 * z + 1, mz - 1);
    size_t sy = (size_t)mx, sz = (size_t)mx * my;
    float s = __ldg(src + x0 + y0 * sy + z0 * sz) + __ldg(src + x1 + y0 * sy + z0 * sz) +
              __ldg(src + x0 + y1 * sy + z0 * sz) + __ldg(src + x1 + y1 * sy + z0 * sz) +
              __ldg(src + x0 + y0 * sy + z1 * sz) + __ldg(src + x1 + y0 * sy + z1 * sz) +
              __ldg(src + x0 + y1 * sy + z1 * sz) + __ldg(src + x1 + y1 * sy + z1 * sz);
    dst[x + (size_t)ox * (y + (size_t)oy * z)] = 0.125f * s;
}

// One thread per fine node, all three components.
__global__ void k_prolong(const float *__restrict__ uc, int cx, int cy, int cz, float *__restrict__ uf, int fx,
                          int fy, int fz, const int *__restrict__ k0x, const int *__restrict__ k0y,
                          const int *__restrict__ k0z, const float *__restrict__ w1x,
                          const float *__restrict__ w1y, const float *__restrict__ w1z)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int z = blockIdx.z;
    if (x >= fx || y >= fy)
        return;
    int kx = k0x[x], ky = k0y[y], kz = k0z[z];
    float wx = w1x[x], wy = w1y[y], wz = w1z[z];
    size_t sy = (size_t)cx, sz = (size_t)cx * cy, ncs = (size_t)cx * cy * cz;
    size_t nfs = (size_t)fx * fy * fz;
    size_t b = kx + ky * sy + kz * sz;
    size_t o = x + (size_t)fx * (y + (size_t)fy * z);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float *u = uc + c * ncs;
        float a0 = lerpf(__ldg(u + b), __ldg(u + b + 1), wx);
        float a1 = lerpf(__ldg(u + b + sy), __ldg(u + b + sy + 1), wx);
        float a2 = lerpf(__ldg(u + b + sz), __ldg(u + b + sz + 1), wx);
        float a3 = lerpf(__ldg(u + b + sz + sy), __ldg(u + b + sz + sy + 1), wx);
        uf[c * nfs + o] = lerpf(lerpf(a0, a1, wy), lerpf(a2, a3, wy), wz);
    }
}

// FP32 -> BF16 (round to nearest even) image copy, float4 reads.
__global__ void __launch_bounds__(256) k_to_bf16(const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst,
                                                 long long n)
{
    const long long n4 = n >> 2;
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n4; e += (long long)gridDim.x * 256) {
        float4 v = reinterpret_cast<const float4 *>(src)[e];
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        reinterpret_cast<__nv_bfloat162 *>(dst)[2 * e] = a;
        reinterpret_cast<__nv_bfloat162 *>(dst)[2 * e + 1] = b;
    }
    if (blockIdx.x == 0 && threadIdx.x < (n & 3))
        dst[4 * n4 + threadIdx.x] = __float2bfloat16_rn(src[4 * n4 + threadIdx.x]);
}

__device__ __forceinline__ void pad_store(float *p, float v) { *p = v; }
__device__ __forceinline__ void pad_store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// Zero-bordered copy of a volume (dims m) into an array of dims m + 4 with the
// volume at offset 2 in every dimension: one thread per element of the
// padded array, so the border is written too.
template <typename TOUT>
__global__ void __launch_bounds__(256) k_pad_template(const float *__restrict__ src, int mx, int my, int mz,
                                                      TOUT *__restrict__ dst)
{
    const int px = mx + 4, py = my + 4;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= px || y >= py)
        return;
    const int sx = x - 2, sy = y - 2, sz = z - 2;
    const bool in = (unsigned)sx < (unsigned)mx && (unsigned)sy < (unsigned)my && (unsigned)sz < (unsigned)mz;
    const float v = in ? __ldg(src + ((size_t)sz * my + sy) * mx + sx) : 0.f;
    pad_store(dst + ((size_t)z * py + y) * px + x, v);
}

// R's normalized gradient field for the fused pass (Eq. 2): R is fixed for the
// whole registration, so its part of every NGF term is formed once per level.
// Per voxel, with b the central-difference gradient of R (the differences
// times 1 / (2 h_c), as the pass forms grad T~): (b / ||b||_rho, rho / ||b||_rho),
// ||b||_rho = sqrt(|b|^2 + rho^2) with a correctly rounded square root and
// division; zero on voxels outside the interior, which Eq. 2's sum leaves out.
// Stored by pairs of columns (x even, x + 1: the two columns a thread of the
// pass holds), 8 floats per pair: bx, bx', by, by' | bz, bz', rho', rho'',
// so that every pair of lanes of the pass's packed arithmetic is one 8-byte
// half of a 16-byte load.  The row length is even, so pair p of a row starts
// at float 8 p and the array has 4 floats per voxel, as a float4 per voxel.
__global__ void k_ref_normal_field(const float *__restrict__ R, int mx, int my, int mz, float hx, float hy, float hz,
                                   float rho, float4 *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= mx || y >= my)
        return;
    const size_t sy = (size_t)mx, sz = (size_t)mx * my;
    const size_t i = x + sy * y + sz * z;
    float o[4] = {0.f, 0.f, 0.f, 0.f};
    if (x >= 1 && x <= mx - 2 && y >= 1 && y <= my - 2 && z >= 1 && z <= mz - 2) {
        const float bx = (__ldg(R + i + 1) - __ldg(R + i - 1)) * hx;
        const float by = (__ldg(R + i + sy) - __ldg(R + i - sy)) * hy;
        const float bz = (__ldg(R + i + sz) - __ldg(R + i - sz)) * hz;
        const float nb = sqrtf(fmaf(bz, bz, fmaf(by, by, bx * bx)) + rho * rho);
        o[0] = bx / nb;
        o[1] = by / nb;
        o[2] = bz / nb;
        o[3] = rho / nb;
    }
    float *pair = reinterpret_cast<float *>(out) + 4 * (i - (x & 1));   // 8 floats of the column pair
#pragma unroll
    for (int c = 0; c < 4; c++)
        pair[2 * c + (x & 1)] = o[c];
}

template <typename TOUT>
cudaError_t launch_pad(const float *src, const int m[3], TOUT *dst, cudaStream_t s)
{
    dim3 blk(32, 8, 1);
    dim3 grd((m[0] + 4 + 31) / 32, (m[1] + 4 + 7) / 8, m[2] + 4);
    k_pad_template<TOUT><<<grd, blk, 0, s>>>(src, m[0], m[1], m[2], dst);
    return cudaGetLastError();
}

}  // namespace

long long padded_voxels(const int m[3]) { return (long long)(m[0] + 4) * (m[1] + 4) * (m[2] + 4); }

cudaError_t launch_pad_template(const float *src, const int m[3], float *dst, cudaStream_t s)
{
    return launch_pad(src, m, dst, s);
}

cudaError_t launch_pad_template(const float *src, const int m[3], __nv_bfloat16 *dst, cudaStream_t s)
{
    return launch_pad(src, m, dst, s);
}

cudaError_t launch_ref_normal_field(const Level &L, double rho, cudaStream_t s)
{
    // the pass's difference factors: 0.5 * (float)(1 / h), as in grad T~
    const LevelGeom g = L.geom();
    dim3 blk(32, 8, 1);
    dim3 grd((L.m[0] + 31) / 32, (L.m[1] + 7) / 8, L.m[2]);
    k_ref_normal_field<<<grd, blk, 0, s>>>(L.R, L.m[0], L.m[1], L.m[2], 0.5f * g.ih[0], 0.5f * g.ih[1],
                                           0.5f * g.ih[2], (float)rho, L.Rn);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float *src, __nv_bfloat16 *dst, long long n, cudaStream_t s)
{
    long long blocks = ((n >> 2) + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    k_to_bf16<<<(int)blocks, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_restrict(const float *src, const int m[3], float *dst, cudaStream_t s)
{
    int o[3] = {(m[0] + 1) / 2, (m[1] + 1) / 2, (m[2] + 1) / 2};
    dim3 blk(32, 8, 1);
    dim3 grd((o[0] + 31) / 32, (o[1] + 7) / 8, o[2]);
    k_restrict<<<grd, blk, 0, s>>>(src, m[0], m[1], m[2], dst, o[0], o[1], o[2]);
    return cudaGetLastError();
}

cudaError_t launch_prolong(const Level &coarse, const Level &fine, const float *uc, float *uf, cudaStream_t s)
{
    dim3 blk(32, 8, 1);
    dim3 grd((fine.n[0] + 31) / 32, (fine.n[1] + 7) / 8, fine.n[2]);
    k_prolong<<<grd, blk, 0, s>>>(uc, coarse.n[0], coarse.n[1], coarse.n[2], uf, fine.n[0], fine.n[1], fine.n[2],
                                  fine.qk0[0], fine.qk0[1], fine.qk0[2], fine.qw1[0], fine.qw1[1], fine.qw1[2]);
    return cudaGetLastError();
}
