// Device code of the fused objective pass for ratio-2 grids: the tile
// pipeline (fused_tile: P, interpolation, NGF residual, adjoint, r and the
// tile's partial P^T sums, optionally the curvature Laplacian of its nodes)
// and the node gather (gather_grad_body: the tile partials of a node plus the
// curvature gradient).  Shared by the single-pair and batched kernels of the
// pass (k_ngf_fused.cu) and the whole-level kernel of small levels
// (k_lbfgs.cu); every includer gets its own internal copies.
#pragma once

#include <type_traits>

#include "batch.h"
#include "internal.h"
#include "ngf_math.cuh"

namespace {

constexpr int BX = 16, BY = 16;                   // threads; each holds two voxel columns
constexpr int CTAS_PER_SM = 2;                    // resident CTAs of the pass per SM
constexpr int NT = BX * BY;                       // 256 threads
constexpr int CW = 2 * BX;                        // voxel columns per tile row, halo included
constexpr int OX = 28, OY = BY - 4;               // output voxels per tile
constexpr int NX = OX / 2 + 1, NY = OY / 2 + 1;   // 15 x 7 node columns per tile
constexpr int NE = 3 * NX * NY;                   // partial entries per node plane (315)
constexpr int PLANE = CW * BY;                    // floats of one shared plane
constexpr int TNX = BX + 1, TNY = BY / 2 + 1;     // node tile of the columns: 17 x 9
constexpr int TNP = 3 * TNY * TNX;                // floats of one node plane tile per array
constexpr int NCOPY = (2 * TNP + NT - 1) / NT;    // node-tile entries copied per thread
constexpr int NCOMB = (TNP + NT - 1) / NT;        // trial node values formed per thread
static_assert(NE <= 2 * NT, "phases D and the curvature take two partial entries per thread");
static_assert(OX == CW - 4 && OY == BY - 4, "the output tile is the thread block less a 2-voxel halo");

// shared layout (floats).  The ring slot of plane z is z & 3 for T~, R and v;
// grad T, written 4 steps before it is read, has a ring of 5 slots taken in
// turn, one per step; node plane K sits in slot K mod node_slots (below).  The rings are
// kept this small so that the CTA's shared memory leaves room for a larger L1,
// which holds the template samples.  RN: the pass reads the normalized
// gradient field of R (a.Rn) into registers and keeps no R ring.
constexpr int GSLOTS = 5;
// node-plane slots: 4 where the tile forms the curvature (plane K - 1 .. K + 1
// read while K + 2 is copied in), else 2 (plane K + 1 read while K + 2 is
// copied in: plane K's values live on in registers)
template <bool CURV>
__host__ __device__ constexpr int node_slots()
{
    return CURV ? 4 : 2;
}
constexpr int RED_PLANE = BY * NX * 3;            // x-reduced rows of one plane [BY][NX][3]
template <bool RN, int NSLOTS>
struct Smem {
    static constexpr int T = 0;                       // T~ ring [4][PLANE]
    static constexpr int R = T + 4 * PLANE;           // R ring [4][PLANE] (without RN: none)
    static constexpr int V = R + (RN ? 0 : 4 * PLANE);   // v ring [4][3][PLANE]
    static constexpr int G = V + 12 * PLANE;          // grad T ring [GSLOTS][3][PLANE]
    static constexpr int RED = G + GSLOTS * 3 * PLANE;   // x-reduced rows [2 steps][RED_PLANE]
    static constexpr int N = RED + 2 * RED_PLANE;     // node planes [NSLOTS][2][TNP] (u or u + t dir, dir)
    static constexpr int FLOATS = N + NSLOTS * 2 * TNP;
    static constexpr size_t BYTES = sizeof(float) * FLOATS;
    static_assert(BYTES <= 227 * 1024, "fused pass exceeds the shared memory of one CTA");
    static_assert((R | V | G | RED | N | PLANE) % 2 == 0, "float2 rows need even offsets");
};
// The single-pair pass over FP32 images of a handle (zero-bordered T) reads R's
// normalized gradient field.  R itself is read by BF16 images (the field would
// undo their memory saving), by the caller's own buffers (no field exists), and
// by the passes that form the curvature too (the batched pass, whose persistent
// kernel has no registers left for the field's prefetch and whose pairs would
// stream 16 bytes per voxel each, and the single-pair form of its arithmetic).
template <typename IMG, bool PAD, bool CURV>
__host__ __device__ constexpr bool reads_rn()
{
    return PAD && !CURV && std::is_same<IMG, float>::value;
}
template <typename IMG, bool PAD, bool CURV>
__host__ __device__ constexpr size_t smem_bytes()
{
    return reads_rn<IMG, PAD, CURV>() ? Smem<true, node_slots<CURV>()>::BYTES : Smem<false, node_slots<CURV>()>::BYTES;
}
template <int NSL>
__device__ __forceinline__ int node_slot(int K)   // K >= -1
{
    return K & (NSL - 1);
}

// The fused kernels' dynamic shared memory, and a carveout preference of just
// that much (with the 1 KB the system reserves per CTA) in percent of the
// SM's 228 KB: the rest of the SM's 256 KB stays L1, where the template's
// samples are cached.
template <typename K>
cudaError_t set_fused_smem(K kernel, size_t bytes)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    const int pct = (int)((100 * CTAS_PER_SM * (bytes + 1024) + 228 * 1024 - 1) / (228 * 1024));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    return e;
}

// 1.5 * 2^23: adding it rounds a float to an integer (the rounding mode picks
// which one); the low bits of the sum then hold that integer plus MAGI
constexpr float MAGF = 12582912.0f;
constexpr int MAGI = 0x4B400000;

// ---- packed FP32 pairs
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    union {
        float2 f;
        unsigned long long u;
    } x, y, d;
    x.f = a;
    y.f = b;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.u) : "l"(x.u), "l"(y.u));
    return d.f;
}
// a + w (b - a), lane by lane: the pair form of lerpf
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float2 w) { return fma2(w, sub2(b, a), a); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// Kahan-compensated pair of running sums
struct KahanF2 {
    float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add(float2 x)
    {
        const float2 y = sub2(x, c);
        const float2 t = add2(s, y);
        c = sub2(sub2(t, s), y);
        s = t;
    }
};

// NGF residual of Eq. 2 for both columns (a = grad T~, b = grad R, 3 pairs
// each): returns psi = 1 - c^2 per lane and writes v = d psi / d a.  psi is
// evaluated through the exact identity
//   (|a|^2 + tau^2)(|b|^2 + rho^2) - (a.b + tau rho)^2 = |a x b|^2 + |tau b - rho a|^2,
// so no cancellation occurs where c is close to 1 (aligned or flat regions).
__device__ __forceinline__ float2 ngf_residual2(const float2 a[3], const float2 b[3], float tau, float rho,
                                                float2 v[3])
{
    const float2 TAU = bc2(tau), RHO = bc2(rho);
    const float2 aa = fma2(a[2], a[2], fma2(a[1], a[1], mul2(a[0], a[0])));
    const float2 bb = fma2(b[2], b[2], fma2(b[1], b[1], mul2(b[0], b[0])));
    const float2 ab = fma2(a[2], b[2], fma2(a[1], b[1], mul2(a[0], b[0])));
    const float2 na2 = add2(aa, bc2(tau * tau)), nb2 = add2(bb, bc2(rho * rho));
    const float2 cx = sub2(mul2(a[1], b[2]), mul2(a[2], b[1]));
    const float2 cy = sub2(mul2(a[2], b[0]), mul2(a[0], b[2]));
    const float2 cz = sub2(mul2(a[0], b[1]), mul2(a[1], b[0]));
    const float2 ex = sub2(mul2(TAU, b[0]), mul2(RHO, a[0]));
    const float2 ey = sub2(mul2(TAU, b[1]), mul2(RHO, a[1]));
    const float2 ez = sub2(mul2(TAU, b[2]), mul2(RHO, a[2]));
    const float2 num = fma2(ez, ez, fma2(ey, ey, fma2(ex, ex, fma2(cz, cz, fma2(cy, cy, mul2(cx, cx))))));
    const float2 den = mul2(na2, nb2);
    const float2 rden = make_float2(__fdividef(1.f, den.x), __fdividef(1.f, den.y));   // approximate: ~2 ulp
    const float2 psi = mul2(num, rden);
    const float2 rs = make_float2(rsqrtf(den.x), rsqrtf(den.y));   // 1 / (||a||_tau ||b||_rho)
    const float2 c = mul2(add2(ab, bc2(tau * rho)), rs);
    const float2 m2c = mul2(bc2(-2.f), c);
    const float2 k1 = mul2(m2c, rs);                                // v = -2c (b / (na nb) - c a / na^2)
    const float2 k2 = mul2(mul2(m2c, c), make_float2(-__fdividef(1.f, na2.x), -__fdividef(1.f, na2.y)));
    v[0] = fma2(k1, b[0], mul2(k2, a[0]));
    v[1] = fma2(k1, b[1], mul2(k2, a[1]));
    v[2] = fma2(k1, b[2], mul2(k2, a[2]));
    return psi;
}

// reciprocal in one MUFU instruction (rcp.approx, max error ~1 ulp; the
// argument is at least tau^2, far above the subnormal range)
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// NGF residual of Eq. 2 for both columns from a = grad T~ (3 pairs) and the
// normalized gradient field of R: bh = b / ||b||_rho and rh = rho / ||b||_rho
// (zero off the interior, where Eq. 2 has no term).  With na2 = |a|^2 + tau^2
// and c' = a . bh + tau rh, the cosine is c = c' / sqrt(na2) and
//   psi = 1 - c^2 = (|a x bh|^2 + |rh a - tau bh|^2) / na2   (no cancellation),
//   v = d psi / d a = -2 (c' / na2) bh + 2 (c' / na2)^2 a,
// so one reciprocal per lane serves both.
__device__ __forceinline__ float2 ngf_residual_rn2(const float2 a[3], const float2 bh[3], float2 rh, float tau,
                                                   float2 v[3])
{
    const float2 TAU = bc2(tau), NTAU = bc2(-tau);
    const float2 aa = fma2(a[2], a[2], fma2(a[1], a[1], mul2(a[0], a[0])));
    const float2 ab = fma2(a[2], bh[2], fma2(a[1], bh[1], mul2(a[0], bh[0])));
    const float2 na2 = add2(aa, bc2(tau * tau));
    const float2 cx = sub2(mul2(a[1], bh[2]), mul2(a[2], bh[1]));
    const float2 cy = sub2(mul2(a[2], bh[0]), mul2(a[0], bh[2]));
    const float2 cz = sub2(mul2(a[0], bh[1]), mul2(a[1], bh[0]));
    const float2 ex = fma2(rh, a[0], mul2(NTAU, bh[0]));
    const float2 ey = fma2(rh, a[1], mul2(NTAU, bh[1]));
    const float2 ez = fma2(rh, a[2], mul2(NTAU, bh[2]));
    const float2 num = fma2(ez, ez, fma2(ey, ey, fma2(ex, ex, fma2(cz, cz, fma2(cy, cy, mul2(cx, cx))))));
    const float2 rna2 = make_float2(rcp_approx(na2.x), rcp_approx(na2.y));
    const float2 psi = mul2(num, rna2);
    const float2 q = mul2(fma2(TAU, rh, ab), rna2);   // c' / na2
    const float2 k1 = mul2(bc2(-2.f), q);
    const float2 k2 = mul2(add2(q, q), q);
    v[0] = fma2(k1, bh[0], mul2(k2, a[0]));
    v[1] = fma2(k1, bh[1], mul2(k2, a[1]));
    v[2] = fma2(k1, bh[2], mul2(k2, a[2]));
    return psi;
}

// 16-byte load of data read once (R's normalized gradient field): through the
// non-coherent path without allocating in L1, which holds the template
// samples.  Predicated inside the instruction (v keeps its value where pred is
// false), so that no branch joins behind it: the load stays in flight until
// its first use a step later.  volatile: it stays where it is issued.
__device__ __forceinline__ void ld_once4(float4 &v, const float4 *p, bool pred)
{
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
        "@q ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%5];\n\t}"
        : "+f"(v.x), "+f"(v.y), "+f"(v.z), "+f"(v.w)
        : "r"((int)pred), "l"(p));
}

__device__ __forceinline__ void cp_async4(float *smem_dst, const float *gsrc, bool valid)
{
    unsigned saddr = (unsigned)__cvta_generic_to_shared(smem_dst);
    int src_size = valid ? 4 : 0;   // 0: no bytes read, the word is zero-filled
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(saddr), "l"(gsrc), "r"(src_size)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ float2 lds2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void sts2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

// One thread's share of the cooperative copy of a node plane (u and, with a
// direction, dir) of the CTA's 17 x 9 node tile: entries tid + q NT.  The
// in-plane offsets do not change along z, so they are computed once.
struct NodeCopy {
    int src[NCOPY];   // offset of the entry's node in plane 0 of u or dir; -1: outside the grid
    int dst[NCOPY];   // entry in a ring slot (>= TNP: the dir tile); -1: no entry
};

template <bool HAS_DIR>
__device__ __forceinline__ NodeCopy node_copy_setup(const LevelGeom &g, int kx0, int ky0, int tid)
{
    const int nn = (int)g.nn, total = (HAS_DIR ? 2 : 1) * TNP;
    NodeCopy nc;
#pragma unroll
    for (int q = 0; q < NCOPY; q++) {
        const int e = tid + q * NT;
        const int r = e >= TNP ? e - TNP : e;
        const int c = r / (TNY * TNX), r2 = r - c * (TNY * TNX);
        const int ly = r2 / TNX, lx = r2 - ly * TNX;
        const int kx = kx0 + lx, ky = ky0 + ly;
        const bool in = e < total && kx >= 0 && kx < g.n[0] && ky >= 0 && ky < g.n[1];
        nc.dst[q] = e < total ? e : -1;
        nc.src[q] = in ? c * nn + kx + g.n[0] * ky : -1;
    }
    return nc;
}

// copy node plane K into its ring slot; nodes outside the grid read as zero
template <int NSL>
__device__ __forceinline__ void issue_node_plane(const NodeCopy &nc, const float *ub, const float *dir,
                                                 float *nodes, int K, int nz, size_t plane_stride)
{
    float *dst = nodes + node_slot<NSL>(K) * 2 * TNP;
    const bool kin = K >= 0 && K < nz;
    const size_t kofs = kin ? plane_stride * (size_t)K : 0;
#pragma unroll
    for (int q = 0; q < NCOPY; q++)
        if (nc.dst[q] >= 0) {
            const bool in = kin && nc.src[q] >= 0;
            const float *base = nc.dst[q] >= TNP ? dir : ub;
            cp_async4(dst + nc.dst[q], in ? base + kofs + nc.src[q] : ub, in);
        }
}

// the trial point of node plane K (copied into its ring slot and visible to
// every thread): u <- u + t dir in place, the same fmaf as the accepted update,
// so the accepted iterate equals the evaluated one bit for bit
template <int NSL>
__device__ __forceinline__ void trial_node_plane(float *nodes, int K, float t, int tid)
{
    float *nu = nodes + node_slot<NSL>(K) * 2 * TNP;
#pragma unroll
    for (int q = 0; q < NCOMB; q++) {
        const int e = tid + q * NT;
        if (e < TNP)
            nu[e] = fmaf(t, nu[e + TNP], nu[e]);
    }
}

// displacement plane K of the thread's two columns from the shared node tile:
// the value at the interval's first node (U, shared) and the bilinear
// interpolation of the in-plane differences (B, x weight 1/4 and 3/4 per lane)
template <int NSL>
__device__ __forceinline__ void column_pair_plane(const float *nodes, int K, int lkx, int lky, float2 WY, float U[3],
                                                  float2 B[3])
{
    const float *nu = nodes + node_slot<NSL>(K) * 2 * TNP;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int o = c * (TNY * TNX) + lky * TNX + lkx;
        const float u00 = nu[o], u10 = nu[o + 1], u01 = nu[o + TNX], u11 = nu[o + TNX + 1];
        const float dx = u10 - u00, dy = u01 - u00, e = (u11 - u00) - dy;
        U[c] = u00;
        const float2 X = make_float2(0.25f * dx, 0.75f * dx);
        const float2 Y = make_float2(fmaf(0.25f, e, dy), fmaf(0.75f, e, dy));
        B[c] = lerp2(X, Y, WY);
    }
}

// image element loads: FP32, or BF16 widened to FP32 (all arithmetic is FP32)
__device__ __forceinline__ float ldimg(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldimg(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
// two adjacent elements starting at an even index (8- or 4-byte aligned)
__device__ __forceinline__ float2 ldimg2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
__device__ __forceinline__ float2 ldimg2(const __nv_bfloat16 *p)
{
    return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162 *>(p)));
}

template <typename IMG>
__device__ __forceinline__ float ldimg_zero_ext(const IMG *T, int mx, int my, int mz, int x, int y, int z)
{
    bool in = (unsigned)x < (unsigned)mx && (unsigned)y < (unsigned)my && (unsigned)z < (unsigned)mz;
    return in ? ldimg(T + (x + mx * (y + my * z))) : 0.f;
}

// Launch order of the tiles: the segment groups of the split by length,
// longest first (so that the short tiles fill the SMs the long ones leave
// free), then segment, then tile column.  Tile id -> (segment s in z order,
// column).
__device__ __forceinline__ void tile_seg_col(const FusedSplit &sp, int ncols, int id, int &s, int &col)
{
    // groups (length, first segment, segments), sorted by length, descending and stable
    int la = sp.l1, sa = 0, ca = sp.n1;
    int lb = sp.l2, sb = sp.n1, cb = sp.n2;
    int lc = sp.lr, sc = sp.n1 + sp.n2, cc = sp.lr > 0 ? 1 : 0;
    auto swap3 = [](int &l0, int &s0, int &c0, int &l1, int &s1, int &c1) {
        int t = l0; l0 = l1; l1 = t;
        t = s0; s0 = s1; s1 = t;
        t = c0; c0 = c1; c1 = t;
    };
    if (lb > la)
        swap3(la, sa, ca, lb, sb, cb);
    if (lc > lb)
        swap3(lb, sb, cb, lc, sc, cc);
    if (lb > la)
        swap3(la, sa, ca, lb, sb, cb);
    int first = sa;
    if (id >= ca * ncols) {
        id -= ca * ncols;
        first = sb;
        if (id >= cb * ncols) {
            id -= cb * ncols;
            first = sc;
        }
    }
    (void)la;
    (void)lc;
    (void)cc;
    const int k = id / ncols;
    s = first + k;
    col = id - k * ncols;
}

// One output tile (launch-order id, see tile_seg_col) of the fused pass; sm is
// the CTA's dynamic shared memory (Smem<RN, NSL>::BYTES).  PAD: a.T is the zero-bordered
// copy of T (dims m + 4, the image at offset 2 in every dimension).  CURV: the
// tile also forms the curvature Laplacian of the nodes it owns (a.w) and their
// share of S (a.partials_S) - where no separate curvature pass can run beside
// this one (the persistent batched grid, the allocation-free call).
template <bool HAS_DIR, typename IMG, bool PAD, bool CURV>
__device__ __forceinline__ void fused_tile(const FusedArgs &a, int tile_id, float *sm)
{
    constexpr bool RN = reads_rn<IMG, PAD, CURV>();
    constexpr int NSL = node_slots<CURV>();
    using SL = Smem<RN, NSL>;
    const LevelGeom &g = a.g;
    // a 16 x 16 block, or 256 threads in one dimension (the whole-level kernel): the same layout
    const int tid = linear_tid(), tx = tid % BX, ty = tid / BX;
    const int sp = 2 * tx + CW * ty;                  // shared-plane index of the thread's first column
    const int ncols = a.ntx * a.nty;
    int seg, col, z0, tz;                             // segment (z order), tile column, its planes
    tile_seg_col(a.split, ncols, tile_id, seg, col);
    a.split.seg(seg, z0, tz);
    const int tile_x = col % a.ntx, tile_y = col / a.ntx;
    const int x0 = tile_x * OX, y0 = tile_y * OY;
    const int xa = x0 - 2 + 2 * tx, y = y0 - 2 + ty;  // the thread's columns: xa (even) and xa + 1
    const int mx = g.m[0], my = g.m[1], mz = g.m[2];
    const int sxy = mx * my;
    // mx is even, so both columns lie inside the image or neither does
    const bool col_in = xa >= 0 && xa < mx && y >= 0 && y < my;
    // t is written by the control phases, within a launch of the whole-level kernel: read through L2
    const float t = HAS_DIR ? (float)__ldcg(a.t_dev) : 0.f;
    // ratio 2: voxel i lies between nodes i/2 and i/2 + 1, weight of the second
    // 1/4 (i even) or 3/4 (i odd); both columns lie in node interval kx0 + tx
    const int lky = ty >> 1;
    const int kx0 = (x0 >> 1) - 1, ky0 = (y0 >> 1) - 1;
    const float2 WY = bc2((y & 1) ? 0.75f : 0.25f);
    const float2 HX = bc2(0.5f * g.ih[0]), HY = bc2(0.5f * g.ih[1]), HZ = bc2(0.5f * g.ih[2]);
    const int zend = z0 + tz;                         // first plane after the segment's output planes
    const size_t tile_lin = (size_t)tile_id;          // this tile's D partial
    // the segment's block of partials: ncols tiles of tz / 2 + 1 node planes
    float *part_tile = a.part + ((size_t)a.split.planes_before(seg) * ncols + (size_t)col * (tz / 2 + 1)) * NE;
    const NodeCopy nc = node_copy_setup<HAS_DIR>(g, kx0, ky0, tid);
    const size_t node_plane = (size_t)g.n[0] * g.n[1];
    const IMG *Tim = static_cast<const IMG *>(a.T);
    const IMG *Rcol = static_cast<const IMG *>(a.R) + (col_in ? xa + mx * y : 0);
    // the pair's two 16-byte halves of R's normalized field (stored by column pair)
    const float4 *Rncol = RN ? a.Rn + (col_in ? xa + mx * y : 0) : nullptr;
    // padded template: row pitch, plane pitch and the largest cell index (padded coordinates)
    const int MXP = mx + 4;
    const int MYP = my + 4;
    const size_t SXYP = (size_t)MXP * MYP;
    const unsigned CXM = (unsigned)mx + 2, CYM = (unsigned)my + 2, CZM = (unsigned)mz + 2;
    constexpr int PADO = PAD ? 2 : 0;                 // image offset inside the template array
    // rows phases B and C run on; output columns (both of the thread's columns)
    const bool rowB = ty >= 1 && ty < BY - 1, rowC = ty >= 2 && ty < BY - 2;
    const bool outxy = rowC && tx >= 1 && tx < BX - 1;
    const bool iny = y >= 1 && y <= my - 2;
    const bool intA = col_in && iny && xa >= 1, intB = col_in && iny && xa + 1 <= mx - 2;
    // lanes of the NGF residual that count: interior voxels (MI), and of those
    // the output columns, whose psi is summed (MO)
    const float2 MI = make_float2(intA ? 1.f : 0.f, intB ? 1.f : 0.f);
    const float2 MO = RN ? bc2(outxy ? 1.f : 0.f)   // psi is zero off the interior
                         : make_float2(intA && outxy ? 1.f : 0.f, intB && outxy ? 1.f : 0.f);
    // rows 0 and BY - 1 (whose v is never read) take their own row for the missing neighbour
    const int dyp = ty < BY - 1 ? CW : 0, dym = ty > 0 ? CW : 0;
    // phase D: partial entries tid and tid + NT = (component, node row jy, node column jx)
    bool dD[2];
    int dofs[2];
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int e = tid + q * NT;
        dD[q] = e < NE;
        const int dc = e / (NX * NY), drem = e - dc * (NX * NY), djy = drem / NX, djx = drem - djy * NX;
        dofs[q] = ((2 * djy) * NX + djx) * 3 + dc;
    }
    // curvature: entries tid and tid + NT = (component, node row, node column) of the
    // node columns this tile owns, local columns 1 .. 14 and rows 1 .. 6 (to 15 and 7 in the
    // last tile column or row) inside the grid; every node has one owner
    int wo[2] = {-1, -1}, wg[2] = {0, 0};   // offset in a node-plane tile (-1: no entry) and in a plane of w
    bool wxy[2] = {false, false};           // node interior in x and y
#pragma unroll
    for (int q = 0; q < 2 && CURV; q++) {
        const int e = tid + q * NT;
        const int dc = e / (NX * NY), drem = e - dc * (NX * NY), ly = drem / NX + 1, lx = drem - (ly - 1) * NX + 1;
        const int kx = kx0 + lx, ky = ky0 + ly;
        const bool own = e < NE && (lx < NX || tile_x == a.ntx - 1) && (ly < NY || tile_y == a.nty - 1) &&
                         kx < g.n[0] && ky < g.n[1];
        wo[q] = own ? dc * (TNY * TNX) + ly * TNX + lx : -1;
        wg[q] = dc * (int)g.nn + kx + g.n[0] * ky;
        wxy[q] = kx >= 1 && kx <= g.n[0] - 2 && ky >= 1 && ky <= g.n[1] - 2;
    }
    float wacc = 0.f;          // sum of w^2 over the entries this thread formed

    float Uhi[3];              // node plane at the top of the current interval (first node)
    float2 Bhi[3];             // its in-plane part, both columns
    float2 fo[3];              // fractional sample coordinates of the interval's odd plane
    int bx0, bx1, by, bz;      // integer bases of the sample cells (with MAGI taken off)
    bool ok0 = true, ok1 = true;   // displacement of the interval representable, per column
    float2 pc[8];              // corners of the next plane, both columns, loaded a step ahead
    float2 fr[3];              // and their fractions
    float2 rnext;              // R of the next plane (without RN)
    float4 bn0 = make_float4(0.f, 0.f, 0.f, 0.f), bn1 = bn0;   // R's normalized field, phase B's next plane (RN)
    float acc_lo[2] = {0.f, 0.f}, hold[2] = {0.f, 0.f};
    KahanF2 psi_sum;
    int gs = 0;                // grad T slot of this step's plane zA; zA - 4 is in slot gs + 1 (mod 5)

    // rows of the x-reduction buffers that no output row writes stay zero
    for (int e = tid; e < 2 * RED_PLANE; e += NT)
        sm[SL::RED + e] = 0.f;

    // ---- A-issue of plane z1: at an even plane (the start of node interval
    // z1 / 2), P on the interval; at an odd plane, the trial values of the node
    // plane copied at the interval start; then the coordinates of plane z1 and
    // the loads of its corners and of R, into registers first used one step later
    auto a_issue = [&](int z1, auto odd_t, bool first) {
        constexpr bool ODD = decltype(odd_t)::value;
        float2 f[3];
        if (!ODD) {
            const int K1 = z1 >> 1;
            float Ulo[3];
            float2 Blo[3];
            if (first) {
                column_pair_plane<NSL>(sm + SL::N, K1, tx, lky, WY, Ulo, Blo);
            } else {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    Ulo[c] = Uhi[c];
                    Blo[c] = Bhi[c];
                }
            }
            column_pair_plane<NSL>(sm + SL::N, K1 + 1, tx, lky, WY, Uhi, Bhi);
            if (first && NSL == 2)
                __syncthreads();   // plane K1's slot takes plane K1 + 2 below (first call: every thread)
            // y-hat = U_lo + lerp(B_lo, (U_hi - U_lo) + B_hi, wz) with wz = 1/4 (even z) or
            // 3/4 (odd z).  The sampling coordinate i + y-hat / h is kept as an integer
            // part plus a small fraction; both depend only on the interval and the
            // parity of z, so they are formed once per interval.
            float q0max = 0.f;
            float2 acc = make_float2(0.f, 0.f);
            int qb[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float ih = g.ih[c];
                const float q0 = Ulo[c] * ih;
                const float qi = floorf(q0);
                const float rem = fmaf(-qi, g.h[c], Ulo[c]);   // |rem| <~ h
                q0max = fmaxf(q0max, fabsf(q0));
                qb[c] = (int)qi;
                const float du = Uhi[c] - Ulo[c];
                const float2 d1 = make_float2(du + Bhi[c].x, du + Bhi[c].y);
                f[c] = mul2(add2(bc2(rem), lerp2(Blo[c], d1, bc2(0.25f))), bc2(ih));
                fo[c] = mul2(add2(bc2(rem), lerp2(Blo[c], d1, bc2(0.75f))), bc2(ih));
                acc = fma2(f[c], f[c], fma2(fo[c], fo[c], acc));
            }
            // every fraction below 1e6 voxels and finite (NaN fails the tests)
            ok0 = q0max < 1.0e6f && acc.x < 1.0e12f;
            ok1 = q0max < 1.0e6f && acc.y < 1.0e12f;
            bx0 = qb[0] + xa + PADO - MAGI;
            bx1 = bx0 + 1;
            by = qb[1] + y + PADO - MAGI;
            bz = qb[2] + z1 + PADO - MAGI;
            // curvature Laplacian of node plane K1 (Sec. 2.1, reading R6): w = L u on
            // interior nodes, 0 elsewhere, from planes K1 - 1 .. K1 + 1 of the ring,
            // for the planes this segment owns (the last segment also its top one)
            if (CURV && K1 >= (z0 >> 1) && (K1 < (zend >> 1) || zend == mz)) {
                const float *pw = sm + SL::N + node_slot<NSL>(K1) * 2 * TNP;
                const float *pm = sm + SL::N + node_slot<NSL>(K1 - 1) * 2 * TNP;
                const float *pp = sm + SL::N + node_slot<NSL>(K1 + 1) * 2 * TNP;
                const bool wz = K1 >= 1 && K1 <= g.n[2] - 2;
                float *wk = a.w + (size_t)K1 * node_plane;
#pragma unroll
                for (int q = 0; q < 2; q++)
                    if (wo[q] >= 0) {
                        const int o = wo[q];
                        float lap = 0.f;
                        if (wxy[q] && wz) {
                            const float u0 = pw[o];
                            lap = fmaf(pw[o + 1] - 2.f * u0 + pw[o - 1], g.iH2[0], lap);
                            lap = fmaf(pw[o + TNX] - 2.f * u0 + pw[o - TNX], g.iH2[1], lap);
                            lap = fmaf(pp[o] - 2.f * u0 + pm[o], g.iH2[2], lap);
                        }
                        wk[wg[q]] = lap;
                        wacc = fmaf(lap, lap, wacc);
                    }
            }
            issue_node_plane<NSL>(nc, a.ub, a.dir, sm + SL::N, K1 + 2, g.n[2], node_plane);
            cp_async_commit();
        } else {
#pragma unroll
            for (int c = 0; c < 3; c++)
                f[c] = fo[c];
            bz += 1;
            if (HAS_DIR)   // copied at the interval start, visible since the last barrier
                trial_node_plane<NSL>(sm + SL::N, (z1 >> 1) + 2, t, tid);
        }
        // integer cells and fractions of both columns: the sum with 1.5 2^23 rounded
        // down holds floor(f) in its low bits
        int ix[2][3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float2 fm = __fadd2_rd(f[c], bc2(MAGF));
            fr[c] = sub2(f[c], sub2(fm, bc2(MAGF)));
            ix[0][c] = __float_as_int(fm.x);
            ix[1][c] = __float_as_int(fm.y);
        }
        const bool zin = col_in && z1 >= 0 && z1 < mz;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const bool okk = k ? ok1 : ok0;
            const int cx = ix[k][0] + (k ? bx1 : bx0), cy = ix[k][1] + by, cz = ix[k][2] + bz;
            float v[8];
            if (PAD) {
                // cells outside [-2, m] (padded [0, m + 2]) move to the far border, whose
                // 8 corners are zeros; so do the columns whose displacement is unusable
                const unsigned ux = okk ? min((unsigned)cx, CXM) : CXM;
                const unsigned uy = min((unsigned)cy, CYM), uz = min((unsigned)cz, CZM);
                const IMG *p = Tim + ((size_t)(uy + (unsigned)MYP * uz) * MXP + ux);
                v[0] = ldimg(p);
                v[1] = ldimg(p + 1);
                v[2] = ldimg(p + MXP);
                v[3] = ldimg(p + MXP + 1);
                v[4] = ldimg(p + SXYP);
                v[5] = ldimg(p + SXYP + 1);
                v[6] = ldimg(p + SXYP + MXP);
                v[7] = ldimg(p + SXYP + MXP + 1);
            } else {
#pragma unroll
                for (int j = 0; j < 8; j++)
                    v[j] = 0.f;
                if (zin && okk) {
                    if ((unsigned)cx < (unsigned)(mx - 1) && (unsigned)cy < (unsigned)(my - 1) &&
                        (unsigned)cz < (unsigned)(mz - 1)) {   // all 8 corners inside
                        const IMG *p = Tim + (cx + mx * (cy + my * cz));
                        v[0] = ldimg(p);
                        v[1] = ldimg(p + 1);
                        v[2] = ldimg(p + mx);
                        v[3] = ldimg(p + mx + 1);
                        v[4] = ldimg(p + sxy);
                        v[5] = ldimg(p + sxy + 1);
                        v[6] = ldimg(p + sxy + mx);
                        v[7] = ldimg(p + sxy + mx + 1);
                    } else {   // zero extension corner by corner
#pragma unroll
                        for (int j = 0; j < 8; j++)
                            v[j] = ldimg_zero_ext(Tim, mx, my, mz, cx + (j & 1), cy + ((j >> 1) & 1),
                                                  cz + (j >> 2));
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 8; j++) {
                if (k)
                    pc[j].y = v[j];
                else
                    pc[j].x = v[j];
            }
        }
        if (!RN)
            rnext = zin ? ldimg2(Rcol + (size_t)sxy * z1) : make_float2(0.f, 0.f);
    };

    // ---- one step of the pipeline; ODD: planes zA + 1 and zA - 5 are odd
    auto step = [&](int s, auto odd_t, auto full_t) {
        constexpr bool FULL = decltype(full_t)::value;   // every phase active: no range tests
        constexpr bool ODD = decltype(odd_t)::value;
        const int zA = z0 - 2 + s;
        // ---- A-finish: T~ and the interpolant differences on plane zA
        if (FULL || zA <= zend + 1) {
            // corners: 0 = (0,0,0), 1 = (1,0,0), 2 = (0,1,0), 3 = (1,1,0), 4..7 the same at z + 1
            const float2 d00 = sub2(pc[1], pc[0]), d10 = sub2(pc[3], pc[2]);
            const float2 d01 = sub2(pc[5], pc[4]), d11 = sub2(pc[7], pc[6]);
            const float2 a00 = fma2(fr[0], d00, pc[0]), a10 = fma2(fr[0], d10, pc[2]);
            const float2 a01 = fma2(fr[0], d01, pc[4]), a11 = fma2(fr[0], d11, pc[6]);
            const float2 e0 = sub2(a10, a00), e1 = sub2(a11, a01);
            const float2 b0 = fma2(fr[1], e0, a00), b1 = fma2(fr[1], e1, a01);
            const float2 gz = sub2(b1, b0);
            const float2 val = fma2(fr[2], gz, b0);
            const float2 gy = lerp2(e0, e1, fr[2]);
            const float2 gx = lerp2(lerp2(d00, d10, fr[1]), lerp2(d01, d11, fr[1]), fr[2]);
            const int slot = zA & 3;
            sts2(sm + SL::T + slot * PLANE + sp, val);
            if (!RN)
                sts2(sm + SL::R + slot * PLANE + sp, rnext);
            float *gq = sm + SL::G + gs * 3 * PLANE + sp;
            sts2(gq, gx);
            sts2(gq + PLANE, gy);
            sts2(gq + 2 * PLANE, gz);
        }
        // ---- A-issue for plane zA + 1
        if (FULL || zA <= zend)
            a_issue(zA + 1, std::integral_constant<bool, ODD>{}, false);
        // ---- B: v on plane zA - 2 (rows 1 .. BY - 2)
        const int zB = zA - 2;
        if constexpr (RN) {
            if (FULL || (zB >= z0 - 1 && zB <= zend)) {
                // R enters through its normalized gradient field, loaded a step ahead
                // (zero off the interior and off the image): no interior tests, and
                // rows 0 and BY - 1, whose v is never read, run the same code
                const int o0 = (zB & 3) * PLANE + sp;
                const float *T0 = sm + SL::T + o0;
                const float2 t0 = lds2(T0);
                const float tl = __shfl_up_sync(0xffffffffu, t0.y, 1, BX);
                const float tr = __shfl_down_sync(0xffffffffu, t0.x, 1, BX);
                const int op = ((zB + 1) & 3) * PLANE + sp, om = ((zB - 1) & 3) * PLANE + sp;
                const float2 typ = lds2(T0 + dyp), tym = lds2(T0 - dym);
                const float2 tzp = lds2(sm + SL::T + op), tzm = lds2(sm + SL::T + om);
                const float2 av[3] = {mul2(make_float2(t0.y - tl, tr - t0.x), HX), mul2(sub2(typ, tym), HY),
                                      mul2(sub2(tzp, tzm), HZ)};
                // the field is stored by column pair: (bx, bx'), (by, by') | (bz, bz'), (rh, rh')
                const float2 bh[3] = {make_float2(bn0.x, bn0.y), make_float2(bn0.z, bn0.w),
                                      make_float2(bn1.x, bn1.y)};
                float2 v[3];
                const float2 psi = ngf_residual_rn2(av, bh, make_float2(bn1.z, bn1.w), a.tau, v);
                if (FULL || (zB >= z0 && zB < zend))
                    psi_sum.add(mul2(psi, MO));
                float *vq = sm + SL::V + (zB & 3) * 3 * PLANE + sp;
                sts2(vq, v[0]);
                sts2(vq + PLANE, v[1]);
                sts2(vq + 2 * PLANE, v[2]);
            }
            // the field at the next step's plane zB + 1, zero off the image.  In a full
            // step that plane lies inside the image and the load depends on the
            // column alone, so a column outside keeps its zeros without a reset
            const int zn = zB + 1;
            const bool ld = col_in && (FULL || (zn >= z0 - 1 && zn <= zend && zn >= 0 && zn < mz));
            if (!FULL)
                bn0 = bn1 = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 *q = Rncol + (size_t)sxy * zn;
            ld_once4(bn0, q, ld);
            ld_once4(bn1, q + 1, ld);
        } else if (FULL || (zB >= z0 - 1 && zB <= zend)) {
            // the pair's own T~ and R (every row), and its x neighbours from the
            // threads beside it: column 2tx - 1 is thread tx - 1's second column,
            // 2tx + 2 thread tx + 1's first (lanes 0 and 31 get their own values;
            // their v is never read)
            const int o0 = (zB & 3) * PLANE + sp;
            const float *T0 = sm + SL::T + o0, *R0 = sm + SL::R + o0;
            const float2 t0 = lds2(T0), r0 = lds2(R0);
            const float tl = __shfl_up_sync(0xffffffffu, t0.y, 1, BX), tr = __shfl_down_sync(0xffffffffu, t0.x, 1, BX);
            const float rl = __shfl_up_sync(0xffffffffu, r0.y, 1, BX), rr = __shfl_down_sync(0xffffffffu, r0.x, 1, BX);
            float2 v[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            if (rowB && (intA || intB) && zB >= 1 && zB <= mz - 2) {
                const int op = ((zB + 1) & 3) * PLANE + sp, om = ((zB - 1) & 3) * PLANE + sp;
                const float2 typ = lds2(T0 + CW), tym = lds2(T0 - CW);
                const float2 tzp = lds2(sm + SL::T + op), tzm = lds2(sm + SL::T + om);
                const float2 ryp = lds2(R0 + CW), rym = lds2(R0 - CW);
                const float2 rzp = lds2(sm + SL::R + op), rzm = lds2(sm + SL::R + om);
                const float2 av[3] = {mul2(make_float2(t0.y - tl, tr - t0.x), HX), mul2(sub2(typ, tym), HY),
                                      mul2(sub2(tzp, tzm), HZ)};
                const float2 bv[3] = {mul2(make_float2(r0.y - rl, rr - r0.x), HX), mul2(sub2(ryp, rym), HY),
                                      mul2(sub2(rzp, rzm), HZ)};
                const float2 psi = ngf_residual2(av, bv, a.tau, a.rho, v);
                v[0] = mul2(v[0], MI);
                v[1] = mul2(v[1], MI);
                v[2] = mul2(v[2], MI);
                if (FULL || (zB >= z0 && zB < zend))
                    psi_sum.add(mul2(psi, MO));
            }
            if (rowB) {
                float *vq = sm + SL::V + (zB & 3) * 3 * PLANE + sp;
                sts2(vq, v[0]);
                sts2(vq + PLANE, v[1]);
                sts2(vq + 2 * PLANE, v[2]);
            }
        }
        // ---- C: r on plane zA - 4 (rows 2 .. BY - 3), x reduction into node columns
        const int zC = zA - 4;
        if (rowC && (FULL || (zC >= z0 && zC < zend))) {   // uniform per warp (a warp holds rows 2w, 2w + 1)
            float2 r[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            // v_x of the pair and of its x neighbours (columns 2tx - 1, 2tx + 2) from the threads beside it
            const float *V0 = sm + SL::V + (zC & 3) * 3 * PLANE + sp;
            const float2 vx = lds2(V0);
            const float vl = __shfl_up_sync(0xffffffffu, vx.y, 1, BX), vr = __shfl_down_sync(0xffffffffu, vx.x, 1, BX);
            if (outxy && col_in && zC < mz) {
                const float *Vzm = sm + SL::V + ((zC - 1) & 3) * 3 * PLANE + 2 * PLANE + sp;
                const float *Vzp = sm + SL::V + ((zC + 1) & 3) * 3 * PLANE + 2 * PLANE + sp;
                const float2 vyp = lds2(V0 + PLANE + CW), vym = lds2(V0 + PLANE - CW);
                const float2 vzm = lds2(Vzm), vzp = lds2(Vzp);
                // adjoint of the central differences (without the factor hbar / 2)
                const float2 gj = fma2(make_float2(vl - vx.y, vx.x - vr), HX,
                                       fma2(sub2(vym, vyp), HY, mul2(sub2(vzm, vzp), HZ)));
                const float *gq = sm + SL::G + (gs == GSLOTS - 1 ? 0 : gs + 1) * 3 * PLANE + sp;
                r[0] = mul2(gj, lds2(gq));
                r[1] = mul2(gj, lds2(gq + PLANE));
                r[2] = mul2(gj, lds2(gq + 2 * PLANE));
            }
            // node column j (0..14) gathers columns 2j .. 2j+3 with weights 1/4, 3/4,
            // 3/4, 1/4: the first two are thread j's pair, the last two thread j+1's
            float *red = sm + SL::RED + (ODD ? 0 : 1) * RED_PLANE + ty * NX * 3;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float lo = fmaf(0.75f, r[c].y, 0.25f * r[c].x), hi = fmaf(0.25f, r[c].y, 0.75f * r[c].x);
                const float nv = lo + __shfl_down_sync(0xffffffffu, hi, 1, BX);
                if (tx < NX)
                    red[tx * 3 + c] = nv;
            }
        }
        // ---- D: y reduction of plane zA - 5 (written last step) and accumulation
        // along z: an even plane gives 3/4 to the lower node plane of its interval
        // and 1/4 to the upper, an odd plane the reverse
        const int zD = zA - 5;
        if (FULL || (zD >= z0 && zD < zend)) {
            const float *red = sm + SL::RED + (ODD ? 1 : 0) * RED_PLANE;
            const int lz = zD - z0;
#pragma unroll
            for (int q = 0; q < 2; q++)
                if (dD[q]) {
                    const float *rp = red + dofs[q];
                    const float v = 0.25f * (rp[0] + rp[3 * NX * 3]) + 0.75f * (rp[NX * 3] + rp[2 * NX * 3]);
                    if (!ODD) {
                        hold[q] = v;
                    } else {
                        const int e = tid + q * NT;
                        part_tile[(size_t)(lz >> 1) * NE + e] = acc_lo[q] + (0.75f * hold[q] + 0.25f * v);
                        acc_lo[q] = 0.25f * hold[q] + 0.75f * v;
                        if (lz == tz - 1)
                            part_tile[(size_t)(tz >> 1) * NE + e] = acc_lo[q];
                    }
                }
        }
        gs = gs == GSLOTS - 1 ? 0 : gs + 1;
        cp_async_wait_all();
        __syncthreads();
    };

    // prologue: node planes of the first interval (and their trial values), then
    // the loads of plane z0 - 2
    {
        const int K0 = (z0 - 2) >> 1;
        issue_node_plane<NSL>(nc, a.ub, a.dir, sm + SL::N, K0, g.n[2], node_plane);
        issue_node_plane<NSL>(nc, a.ub, a.dir, sm + SL::N, K0 + 1, g.n[2], node_plane);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        if (HAS_DIR) {
            trial_node_plane<NSL>(sm + SL::N, K0, t, tid);
            trial_node_plane<NSL>(sm + SL::N, K0 + 1, t, tid);
            __syncthreads();
        }
        a_issue(z0 - 2, std::false_type{}, true);
        cp_async_wait_all();
        __syncthreads();
    }

    // z0 is even: zA + 1 is odd on even steps
    const int nsteps = tz + 7;
    // steps s and s + 1 in turn (z0 is even: zA + 1 is odd on even steps); from
    // step 7 to step tz + 2 every phase is active, and those steps run without
    // the range tests, so the phases of a step form one block of code the
    // compiler can interleave
    int s = 0;
    for (; s < 8 && s < nsteps; s += 2) {
        step(s, std::true_type{}, std::false_type{});
        if (s + 1 < nsteps)
            step(s + 1, std::false_type{}, std::false_type{});
    }
    for (; s + 1 <= tz + 2; s += 2) {
        step(s, std::true_type{}, std::true_type{});
        step(s + 1, std::false_type{}, std::true_type{});
    }
    for (; s < nsteps; s += 2) {
        step(s, std::true_type{}, std::false_type{});
        if (s + 1 < nsteps)
            step(s + 1, std::false_type{}, std::false_type{});
    }
    const float2 ps = psi_sum.s;
    const double ssum = block_sum_to_f64(ps.x + ps.y, reinterpret_cast<double *>(sm + SL::RED));
    if (tid == 0)
        a.partials[tile_lin] = ssum;
    if (CURV) {
        const double wsum = block_sum_to_f64(wacc, reinterpret_cast<double *>(sm + SL::RED));
        if (tid == 0)
            a.partials_S[tile_lin] = wsum;
    }
}

// Segment (z order) and local node plane of node plane kz: the segment whose
// planes z0 / 2 .. (z0 + len) / 2 - 1 contain it, or the last segment for the
// last node plane.
__device__ __forceinline__ void node_seg(const FusedSplit &sp, int kz, int &s, int &jz)
{
    const int h1 = sp.l1 / 2, h2 = sp.l2 / 2;
    const int e1 = sp.n1 * h1, e2 = e1 + sp.n2 * h2;
    if (kz < e1) {
        s = kz / h1;
        jz = kz - s * h1;
    } else if (kz < e2) {
        const int i = (kz - e1) / h2;
        s = sp.n1 + i;
        jz = kz - e1 - i * h2;
    } else if (sp.lr > 0) {
        s = sp.n1 + sp.n2;
        jz = kz - e2;
    } else {
        s = sp.count() - 1;
        int z0, len;
        sp.seg(s, z0, len);
        jz = kz - z0 / 2;
    }
}

// grad J at node k = sum of the tile partials that contain k (P^T r) plus
// alpha hbar_y L^T w (curvature), one thread per node, 3 components.  A block
// takes GATHER_NODES consecutive nodes of one node plane (bx-th run of plane
// kz), so that no lane idles at the end of a row.  Along x and y the node's
// owner tile column is t = min(k / (o/2), nt - 1) at local index
// j = k - (o/2) t; when j = 0 and t > 0 the lower column also holds it, at
// j = o/2.  Along z its owner is the segment holding its node plane
// (node_seg); at the segment's first plane the previous segment also holds it,
// at its last plane.  The up to 8 partials are added owner first, lower x
// before lower y before lower z.  Every thread of the block calls it (it has
// block barriers).  FRESH: the partials and w were written earlier in the same
// launch (the whole-level kernel), so they are read through L2, not the
// read-only path, whose lines may predate them.
template <bool FRESH = false>
__device__ __forceinline__ float ld_part(const float *p)
{
    return FRESH ? __ldcg(p) : __ldg(p);
}
template <bool FRESH = false>
__device__ __forceinline__ void gather_grad_body(const LevelGeom &g, const float *__restrict__ part,
                                                 const FusedSplit &sp, int ntx, int nty,
                                                 const float *__restrict__ w, float alpha_hy,
                                                 float *__restrict__ grad, int bx, int kz)
{
    // the plane's z bookkeeping, the same for the whole block: the owner
    // segment's partial plane and tile-column stride, and the previous
    // segment's when it also holds the plane
    __shared__ long long s_zo, s_zl;
    __shared__ int s_so, s_sl;
    if (threadIdx.x == 0) {
        int so, jz, z0, len;
        node_seg(sp, kz, so, jz);
        const long long ncols = (long long)ntx * nty;
        sp.seg(so, z0, len);
        s_so = (len / 2 + 1) * NE;
        s_zo = sp.planes_before(so) * ncols * NE + (long long)jz * NE;
        s_sl = 0;
        s_zl = -1;
        if (jz == 0 && so > 0) {
            sp.seg(so - 1, z0, len);
            s_sl = (len / 2 + 1) * NE;
            s_zl = sp.planes_before(so - 1) * ncols * NE + (long long)(len / 2) * NE;
        }
    }
    __syncthreads();
    const long long zo = s_zo, zl = s_zl;
    const int stride_o = s_so, stride_l = s_sl;
    __syncthreads();   // a caller's next block item may overwrite them
    const int n0 = g.n[0], n01 = g.n[0] * g.n[1];
    const int i = bx * GATHER_NODES + threadIdx.x;   // node of the plane
    if (i >= n01)
        return;   // (after the barriers: a caller's barrier after it is still reached)
    // ky = i / n0: a float estimate, exact after one correction either way
    int ky = (int)((float)i * __frcp_rn((float)n0));
    int kx = i - ky * n0;
    if (kx < 0) {
        ky--;
        kx += n0;
    } else if (kx >= n0) {
        ky++;
        kx -= n0;
    }
    const int tx = min(kx / (NX - 1), ntx - 1), ty = min(ky / (NY - 1), nty - 1);
    const int jx = kx - (NX - 1) * tx, jy = ky - (NY - 1) * ty;
    const bool lx = jx == 0 && tx > 0, ly = jy == 0 && ty > 0, lz = zl >= 0;
    const long long col = tx + (long long)ntx * ty;
    const float *po = part + zo + col * stride_o + (jy * NX + jx);
    const float *pl = lz ? part + zl + col * stride_l + (jy * NX + jx) : po;
    float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const bool ux = q & 1, uy = (q >> 1) & 1, uz = q >> 2;
        if ((ux && !lx) || (uy && !ly) || (uz && !lz))
            continue;
        const long long stride = uz ? stride_l : stride_o;
        // the lower column's copy: one column back, local index o/2 instead of 0
        const float *p = (uz ? pl : po) + (ux ? -stride + (NX - 1) : 0) + (uy ? -stride * ntx + (NY - 1) * NX : 0);
        s[0] += ld_part<FRESH>(p);
        s[1] += ld_part<FRESH>(p + NX * NY);
        s[2] += ld_part<FRESH>(p + 2 * NX * NY);
    }
    // the pass leaves out the factor hbar / 2 of the adjoint and 1 / h_c of the
    // interpolant gradient: component c of P^T r is hbar / (2 h_c) times the sum
    const float hh = 0.5f * g.hbar;
    const float sc[3] = {hh * g.ih[0], hh * g.ih[1], hh * g.ih[2]};
    const int k = i + n01 * kz;
    const int st[3] = {1, n0, n01};
    const int j[3] = {kx, ky, kz};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float *wc = w + c * g.nn;
        const float w0 = ld_part<FRESH>(wc + k);
        float l = 0.f;
#pragma unroll
        for (int e = 0; e < 3; e++) {
            const float lo = j[e] > 0 ? ld_part<FRESH>(wc + k - st[e]) : 0.f;
            const float hi = j[e] < g.n[e] - 1 ? ld_part<FRESH>(wc + k + st[e]) : 0.f;
            l = fmaf(lo + hi - 2.f * w0, g.iH2[e], l);
        }
        grad[c * g.nn + k] = fmaf(alpha_hy, l, sc[c] * s[c]);
    }
}

}  // namespace
