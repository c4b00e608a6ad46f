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

__device__ __forceinline__ int linear_bid()
{
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// Block sum of one float per thread: FP32 within each warp (32 terms), FP64
// across warps.  The result is valid in thread 0.  sm holds >= nwarps doubles.
__device__ __forceinline__ double block_sum_to_f64(float v, double *sm)
{
    const int tid = linear_tid();
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    v = warp_sum(v);
    if ((tid & 31) == 0)
        sm[tid >> 5] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < (nthreads + 31) / 32; w++)
            s += sm[w];
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
