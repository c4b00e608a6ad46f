// Shared device-side definitions of the CUDA path (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define REG_WARP 32

// Geometry of one pyramid level as seen by the kernels (passed by value).
// Per-dimension tables implement the grid conversion P and its adjoint with
// weights and index sets determined beforehand, one dimension at a time
// (Sec. 2.2 "Grid conversion", Eq. 3).
struct LevelGeom {
    int m[3];            // image voxels
    int n[3];            // deformation nodes
    float h[3];          // voxel spacing (mm)
    float ih[3];         // 1 / h
    float iH2[3];        // 1 / H^2 (node spacing)
    float hbar;          // h_x h_y h_z
    float hbar_y;        // H_x H_y H_z
    long long nv;        // voxels
    long long nn;        // nodes
    // P: voxel index i_d -> first node k0 and weight of node k0 + 1
    const int *pk0[3];
    const float *pw1[3];
    // P^T: node index k_d -> first voxel, voxel count, weights [k * tmaxw + j]
    const int *tfirst[3];
    const int *tcnt[3];
    const float *tw[3];
    int tmaxw[3];
};

__device__ __forceinline__ float lerpf(float a, float b, float w) { return fmaf(w, b - a, a); }

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ int linear_tid()
{
    return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}

__device__ __forceinline__ int nthreads() { return blockDim.x * blockDim.y * blockDim.z; }

__device__ __forceinline__ int linear_bid()
{
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// Block sum of one float per thread, returned as FP64 in thread 0 (other
// threads: 0).  sm holds >= nwarps floats (declared double for callers).
__device__ __forceinline__ double block_sum_to_f64(float v, double *sm)
{
    // FP32 inside the block (warp sums, then the warp totals by one warp, in a
    // fixed order); the block total goes to FP64 for the cross-block sum.  FP64
    // arithmetic costs ~64 cycles per warp instruction on this GPU, so it is
    // kept to the cross-block step.
    float *smf = reinterpret_cast<float *>(sm);
    const int tid = linear_tid();
    const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) / 32;
    v = warp_sum(v);
    if ((tid & 31) == 0)
        smf[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid < 32) {
        float x = warp_sum(tid < nw ? smf[tid] : 0.f);
        if (tid == 0)
            s = (double)x;
    }
    __syncthreads();
    return s;
}

// Kahan-compensated FP32 accumulator for per-thread running sums.
struct KahanF {
    float s, c;
    __device__ __forceinline__ KahanF() : s(0.f), c(0.f) {}
    __device__ __forceinline__ void add(float x)
    {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Double-float sums: a value as an unevaluated pair hi + lo of FP32 numbers
// with |lo| <= ulp(hi) / 2, added with Knuth's two-sum (exact error of one
// addition) and renormalised with Dekker's fast two-sum.  About 48 bits of
// significand at the cost of a few FP32 instructions: on this GPU an FP64
// instruction costs about 64 issue cycles, so sums on the critical path of a
// control phase run faster as double-float than as FP64.  The order of the
// additions is fixed by the callers, so the sums are deterministic.
struct DFloat {
    float hi, lo;
};
__device__ __forceinline__ DFloat df_renorm(float s, float e)
{
    const float hi = s + e;
    return DFloat{hi, e - (hi - s)};
}
__device__ __forceinline__ DFloat df_add(DFloat a, DFloat b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return df_renorm(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ DFloat df_add(DFloat a, float b) { return df_add(a, DFloat{b, 0.f}); }
__device__ __forceinline__ double df_to_double(DFloat a) { return (double)a.hi + (double)a.lo; }

// Ordered FP64 sum (is_max: max) of count values x[i0], x[i0 + step], ...,
// starting from s.  The loads go out 8 at a time so that their L2 round trips
// overlap; the additions keep the index order, so the result is the plain
// sequential one.
__device__ __forceinline__ double ordered_reduce(const double *__restrict__ x, long long i0, int count,
                                                 long long step, bool is_max, double s)
{
    for (int k0 = 0; k0 < count; k0 += 8) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; k++)
            v[k] = k0 + k < count ? __ldcg(x + i0 + (long long)(k0 + k) * step) : 0.0;
#pragma unroll
        for (int k = 0; k < 8; k++)
            if (k0 + k < count)
                s = is_max ? fmax(s, v[k]) : s + v[k];
    }
    return s;
}

// Deterministic FP64 sum of block partials: scal = [J, D, S].  The summation
// order is a fixed 512-wide layout (strided sums, then a halving tree), the
// same for any block size, so every kernel that ends an evaluation with it
// gets bit-identical scalars.
__device__ __forceinline__ void finalize_body(const double *__restrict__ pD, int nD, const double *__restrict__ pS,
                                              int nS, double hbar_half, double alpha, double hy_half,
                                              double *__restrict__ scal)
{
    __shared__ double sd[512], ss[512];
    const int t = linear_tid(), nt = nthreads();
    for (int v = t; v < 512; v += nt) {
        sd[v] = ordered_reduce(pD, v, v < nD ? (nD - v + 511) / 512 : 0, 512, false, 0.0);
        ss[v] = ordered_reduce(pS, v, v < nS ? (nS - v + 511) / 512 : 0, 512, false, 0.0);
    }
    __syncthreads();
    for (int o = 256; o > 0; o >>= 1) {
        for (int v = t; v < o; v += nt) {
            sd[v] += sd[v + o];
            ss[v] += ss[v + o];
        }
        __syncthreads();
    }
    if (t == 0) {
        double D = hbar_half * sd[0], S = hy_half * ss[0];
        scal[0] = D + alpha * S;
        scal[1] = D;
        scal[2] = S;
    }
}
