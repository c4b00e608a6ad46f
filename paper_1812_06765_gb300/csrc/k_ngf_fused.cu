// Fused objective pass for ratio-2 grids (every image dimension even and
// n_d = m_d / 2 + 1, the default rule): one kernel computes, per voxel,
//   y-hat = P u (Eq. 1), T(x + y-hat) and its interpolant gradient,
//   the NGF residual of Eq. 2 and v = d psi / d grad T,
//   g = adjoint central difference of v, r = g grad T (the chain rule),
// and reduces r to per-tile partial node sums of P^T r (Eq. 3); a second,
// node-parallel kernel adds up the (at most 8) tile partials of each node and
// the curvature gradient.  Nothing per voxel goes to HBM.
//
// Tiling.  A CTA of 16 x 32 threads owns a 32 x 32 block of voxel columns:
// thread (tx, ty) holds the two adjacent columns 2 tx and 2 tx + 1 of row ty.
// The inner 28 x 28 columns are the output tile; the 2-voxel halo is what the
// stencil chain T~ -> a -> v -> g reaches.  The CTA marches along z through a
// segment of TZ output planes.  With ratio 2 the P weights are 1/4 and 3/4;
// tiles start at even x, so the two columns of a thread always lie in the
// same node interval (x weights 1/4 and 3/4 of the same nodes), and the node
// loads, P's integer cell and the x reduction of P^T are shared by the pair.
// A node gathers voxels 2k-2 .. 2k+1 with weights 1/4, 3/4, 3/4, 1/4 per
// dimension, so an output tile of 28 x 28 x TZ voxels feeds 15 x 15 x
// (TZ/2 + 1) nodes; neighbouring tiles share one node plane per dimension and
// the gather kernel sums them.
//
// Pipeline.  Step s works on plane zA = z0 - 2 + s and the lagging planes
//   A-finish zA    : interpolate T at both columns from the corners loaded
//                    last step
//   A-issue  zA+1  : at the first plane of a node interval, P on the interval
//                    (both planes) and the cp.async of the node-plane tile two
//                    intervals ahead; the coordinates of plane zA+1 and the
//                    loads of its 2 x 8 corners and of R into registers, first
//                    used one step later
//   B  zA-2        : v from T~ and R planes zA-3 .. zA-1
//   C  zA-4        : r from v planes zA-5 .. zA-3; x reduction to node columns
//   D  zA-5        : y reduction of last step's rows, accumulation along z
// Every phase reads only what earlier steps wrote, so one barrier per step
// suffices, and the global loads of a plane overlap a whole step of compute.
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <queue>
#include <type_traits>
#include <vector>

#include "batch.h"
#include "internal.h"
#include "lbfgs_control.cuh"
#include "ngf_math.cuh"

namespace {

constexpr int BX = 16, BY = 32;                   // threads; each holds two voxel columns
constexpr int NT = BX * BY;                       // 512 threads
constexpr int CW = 2 * BX;                        // voxel columns per tile row, halo included
constexpr int OX = 28, OY = 28;                   // output voxels per tile
constexpr int NX = OX / 2 + 1, NY = OY / 2 + 1;   // 15 x 15 node columns per tile
constexpr int NE = 3 * NX * NY;                   // partial entries per node plane (675)
constexpr int PLANE = CW * BY;                    // floats of one shared plane
constexpr int TNX = BX + 1, TNY = BY / 2 + 1;     // node tile of the columns: 17 x 17
constexpr int TNP = 3 * TNY * TNX;                // floats of one node plane tile per array
constexpr int NCOPY = (2 * TNP + NT - 1) / NT;    // node-tile entries copied per thread

// shared layout (floats); the ring slot of plane z is z & 3 (z & 7 for grad T)
constexpr int OFF_T = 0;                          // T~ ring [4][PLANE]
constexpr int OFF_R = OFF_T + 4 * PLANE;          // R ring [4][PLANE]
constexpr int OFF_V = OFF_R + 4 * PLANE;          // v ring [4][3][PLANE]
constexpr int OFF_G = OFF_V + 12 * PLANE;         // grad T ring [8][3][PLANE]
constexpr int RED_PLANE = BY * NX * 3;            // x-reduced rows of one plane [BY][NX][3]
constexpr int OFF_RED = OFF_G + 24 * PLANE;       // x-reduced rows [2 steps][RED_PLANE]
constexpr int OFF_N = OFF_RED + 2 * RED_PLANE;    // node planes [4][2][TNP] (u, dir)
constexpr int SMEM_FLOATS = OFF_N + 4 * 2 * TNP;
constexpr size_t SMEM_BYTES = sizeof(float) * SMEM_FLOATS;
static_assert(SMEM_BYTES <= 227 * 1024, "fused pass exceeds the shared memory of one CTA");
static_assert((OFF_R | OFF_V | OFF_G | OFF_RED | OFF_N | PLANE) % 2 == 0, "float2 rows need even offsets");


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
__device__ __forceinline__ void sts2(float *p, float a, float b) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }

// One thread's share of the cooperative copy of a node plane (u and, with a
// direction, dir) of the CTA's 17 x 17 node tile: entries tid + q NT.  The
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

// copy node plane K into ring slot K & 3; nodes outside the grid read as zero
__device__ __forceinline__ void issue_node_plane(const NodeCopy &nc, const float *ub, const float *dir, float *sm,
                                                 int K, int nz, size_t plane_stride)
{
    float *dst = sm + OFF_N + (K & 3) * 2 * TNP;
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

// displacement plane K of the thread's two columns from the shared node tile:
// the value at the interval's first node (U, shared) and the bilinear
// interpolation of the in-plane differences (Bd, x weight 1/4 and 3/4)
template <bool HAS_DIR>
__device__ __forceinline__ void column_pair_plane(const float *sm, int K, int lkx, int lky, float wy, float t,
                                                  float U[3], float Bd[2][3])
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
        const float dx = u10 - u00, dy = u01 - u00, dxy = u11 - u00;
        U[c] = u00;
        Bd[0][c] = lerpf(0.25f * dx, lerpf(dy, dxy, 0.25f), wy);
        Bd[1][c] = lerpf(0.75f * dx, lerpf(dy, dxy, 0.75f), wy);
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
// the CTA's dynamic shared memory (SMEM_BYTES).
template <bool HAS_DIR, typename IMG>
__device__ __forceinline__ void fused_tile(const FusedArgs &a, int tile_id, float *sm)
{
    const LevelGeom &g = a.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
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
    const float t = HAS_DIR ? (float)__ldg(a.t_dev) : 0.f;
    // ratio 2: voxel i lies between nodes i/2 and i/2 + 1, weight of the second
    // 1/4 (i even) or 3/4 (i odd); both columns lie in node interval kx0 + tx
    const int lky = ty >> 1;
    const int kx0 = (x0 >> 1) - 1, ky0 = (y0 >> 1) - 1;
    const float wy = (y & 1) ? 0.75f : 0.25f;
    const float hx = 0.5f * g.ih[0], hy = 0.5f * g.ih[1], hz = 0.5f * g.ih[2];
    const float half_hbar = 0.5f * g.hbar;
    const int zend = z0 + tz;                         // first plane after the segment's output planes
    const size_t tile_lin = (size_t)tile_id;          // this tile's D partial
    // the segment's block of partials: ncols tiles of tz / 2 + 1 node planes
    float *part_tile = a.part + ((size_t)a.split.planes_before(seg) * ncols + (size_t)col * (tz / 2 + 1)) * NE;
    const NodeCopy nc = node_copy_setup<HAS_DIR>(g, kx0, ky0, tid);
    const size_t node_plane = (size_t)g.n[0] * g.n[1];
    const IMG *Tim = static_cast<const IMG *>(a.T);
    const IMG *Rcol = static_cast<const IMG *>(a.R) + (col_in ? xa + mx * y : 0);
    // rows phases B and C run on; output columns (both of the thread's columns)
    const bool rowB = ty >= 1 && ty < BY - 1, rowC = ty >= 2 && ty < BY - 2;
    const bool outxy = rowC && tx >= 1 && tx < BX - 1;
    const bool iny = y >= 1 && y <= my - 2;
    const bool intA = col_in && iny && xa >= 1, intB = col_in && iny && xa + 1 <= mx - 2;
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

    float Uhi[3], Bhi[2][3];   // node plane at the top of the current interval, both columns
    float fo[2][3];            // fractions of the interval's odd plane
    int qb[3];                 // integer part of y-hat / h on the interval
    bool iv_ok[2];             // displacement of the interval representable
    float pc[2][8], fr[2][3];  // corners and fractions of the next plane, loaded a step ahead
    float2 rnext;              // R of the next plane
    float acc_lo[2] = {0.f, 0.f}, hold[2] = {0.f, 0.f};
    KahanF psi_sum;

    // rows of the x-reduction buffers that no output row writes stay zero
    for (int e = tid; e < 2 * RED_PLANE; e += NT)
        sm[OFF_RED + e] = 0.f;

    // ---- A-issue of plane z1: at an even plane (the start of node interval
    // z1 / 2), P on the interval; then the coordinates of plane z1 and the
    // loads of its corners and of R, into registers first used one step later
    auto a_issue = [&](int z1, auto odd_t, bool first) {
        constexpr bool ODD = decltype(odd_t)::value;
        float f[2][3];
        if (!ODD) {
            const int K1 = z1 >> 1;
            float Ulo[3], Blo[2][3];
            if (first) {
                column_pair_plane<HAS_DIR>(sm, K1, tx, lky, wy, t, Ulo, Blo);
            } else {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    Ulo[c] = Uhi[c];
                    Blo[0][c] = Bhi[0][c];
                    Blo[1][c] = Bhi[1][c];
                }
            }
            column_pair_plane<HAS_DIR>(sm, K1 + 1, tx, lky, wy, t, Uhi, Bhi);
            // y-hat = U_lo + lerp(B_lo, (U_hi - U_lo) + B_hi, wz) with wz = 1/4 (even z) or
            // 3/4 (odd z).  The sampling coordinate i + y-hat / h is kept as an integer
            // part plus a small fraction; both depend only on the interval and the
            // parity of z, so they are formed once per interval.
            iv_ok[0] = iv_ok[1] = true;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float ih = g.ih[c];
                const float q0 = Ulo[c] * ih;
                const float qi = floorf(q0);
                const float rem = fmaf(-qi, g.h[c], Ulo[c]);   // |rem| <~ h
                qb[c] = (int)qi;
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    const float d1 = (Uhi[c] - Ulo[c]) + Bhi[k][c];
                    iv_ok[k] = iv_ok[k] && fabsf(q0) < 1.0e6f && fabsf(Blo[k][c] * ih) < 1.0e6f &&
                               fabsf(d1 * ih) < 1.0e6f;
                    f[k][c] = (rem + lerpf(Blo[k][c], d1, 0.25f)) * ih;
                    fo[k][c] = (rem + lerpf(Blo[k][c], d1, 0.75f)) * ih;
                }
            }
            issue_node_plane(nc, a.ub, a.dir, sm, K1 + 2, g.n[2], node_plane);
            cp_async_commit();
        } else {
#pragma unroll
            for (int k = 0; k < 2; k++)
#pragma unroll
                for (int c = 0; c < 3; c++)
                    f[k][c] = fo[k][c];
        }
        const bool zin = col_in && z1 >= 0 && z1 < mz;
#pragma unroll
        for (int k = 0; k < 2; k++) {
#pragma unroll
            for (int j = 0; j < 8; j++)
                pc[k][j] = 0.f;
            int cc[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float fl = floorf(f[k][c]);
                fr[k][c] = f[k][c] - fl;
                cc[c] = qb[c] + (int)fl;
            }
            const int cx = cc[0] + xa + k, cy = cc[1] + y, cz = cc[2] + z1;
            if (zin && iv_ok[k]) {
                if ((unsigned)cx < (unsigned)(mx - 1) && (unsigned)cy < (unsigned)(my - 1) &&
                    (unsigned)cz < (unsigned)(mz - 1)) {   // all 8 corners inside
                    const IMG *p = Tim + (cx + mx * (cy + my * cz));
                    pc[k][0] = ldimg(p);
                    pc[k][1] = ldimg(p + 1);
                    pc[k][2] = ldimg(p + mx);
                    pc[k][3] = ldimg(p + mx + 1);
                    pc[k][4] = ldimg(p + sxy);
                    pc[k][5] = ldimg(p + sxy + 1);
                    pc[k][6] = ldimg(p + sxy + mx);
                    pc[k][7] = ldimg(p + sxy + mx + 1);
                } else {   // zero extension corner by corner
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        pc[k][j] = ldimg_zero_ext(Tim, mx, my, mz, cx + (j & 1), cy + ((j >> 1) & 1), cz + (j >> 2));
                }
            }
        }
        rnext = zin ? ldimg2(Rcol + (size_t)sxy * z1) : make_float2(0.f, 0.f);
    };

    // ---- one step of the pipeline; ODD: planes zA + 1 and zA - 5 are odd
    auto step = [&](int s, auto odd_t) {
        constexpr bool ODD = decltype(odd_t)::value;
        const int zA = z0 - 2 + s;
        // ---- A-finish: T~ and grad T on plane zA
        if (zA <= zend + 1) {
            float val[2], gx[2], gy[2], gz[2];
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const float t000 = pc[k][0], t100 = pc[k][1], t010 = pc[k][2], t110 = pc[k][3];
                const float t001 = pc[k][4], t101 = pc[k][5], t011 = pc[k][6], t111 = pc[k][7];
                const float f0 = fr[k][0], f1 = fr[k][1], f2 = fr[k][2];
                const float a00 = lerpf(t000, t100, f0), a10 = lerpf(t010, t110, f0);
                const float a01 = lerpf(t001, t101, f0), a11 = lerpf(t011, t111, f0);
                const float b0 = lerpf(a00, a10, f1), b1 = lerpf(a01, a11, f1);
                val[k] = lerpf(b0, b1, f2);
                const float dx0 = lerpf(t100 - t000, t110 - t010, f1), dx1 = lerpf(t101 - t001, t111 - t011, f1);
                gx[k] = lerpf(dx0, dx1, f2) * g.ih[0];
                gy[k] = lerpf(a10 - a00, a11 - a01, f2) * g.ih[1];
                gz[k] = (b1 - b0) * g.ih[2];
            }
            const int slot = zA & 3;
            sts2(sm + OFF_T + slot * PLANE + sp, val[0], val[1]);
            sts2(sm + OFF_R + slot * PLANE + sp, rnext.x, rnext.y);
            float *gq = sm + OFF_G + (zA & 7) * 3 * PLANE + sp;
            sts2(gq, gx[0], gx[1]);
            sts2(gq + PLANE, gy[0], gy[1]);
            sts2(gq + 2 * PLANE, gz[0], gz[1]);
        }
        // ---- A-issue for plane zA + 1
        if (zA <= zend)
            a_issue(zA + 1, std::integral_constant<bool, ODD>{}, false);
        // ---- B: v on plane zA - 2 (rows 1 .. 30)
        const int zB = zA - 2;
        if (zB >= z0 - 1 && zB <= zend) {
            // the pair's own T~ and R (every row), and its x neighbours from the
            // threads beside it: column 2tx - 1 is thread tx - 1's second column,
            // 2tx + 2 thread tx + 1's first (lanes 0 and 31 get their own values;
            // their v is never read)
            const int o0 = (zB & 3) * PLANE + sp;
            const float *T0 = sm + OFF_T + o0, *R0 = sm + OFF_R + o0;
            const float2 t0 = lds2(T0), r0 = lds2(R0);
            const float tl = __shfl_up_sync(0xffffffffu, t0.y, 1, BX), tr = __shfl_down_sync(0xffffffffu, t0.x, 1, BX);
            const float rl = __shfl_up_sync(0xffffffffu, r0.y, 1, BX), rr = __shfl_down_sync(0xffffffffu, r0.x, 1, BX);
            float va[3] = {0.f, 0.f, 0.f}, vb[3] = {0.f, 0.f, 0.f};
            if (rowB && (intA || intB) && zB >= 1 && zB <= mz - 2) {
                const int op = ((zB + 1) & 3) * PLANE + sp, om = ((zB - 1) & 3) * PLANE + sp;
                const float2 typ = lds2(T0 + CW), tym = lds2(T0 - CW);
                const float2 tzp = lds2(sm + OFF_T + op), tzm = lds2(sm + OFF_T + om);
                const float2 ryp = lds2(R0 + CW), rym = lds2(R0 - CW);
                const float2 rzp = lds2(sm + OFF_R + op), rzm = lds2(sm + OFF_R + om);
                const bool out = outxy && zB >= z0 && zB < zend;
                if (intA) {
                    const float av[3] = {(t0.y - tl) * hx, (typ.x - tym.x) * hy, (tzp.x - tzm.x) * hz};
                    const float bv[3] = {(r0.y - rl) * hx, (ryp.x - rym.x) * hy, (rzp.x - rzm.x) * hz};
                    const float psi = ngf_residual(av, bv, a.tau, a.rho, va);
                    if (out)
                        psi_sum.add(psi);
                }
                if (intB) {
                    const float av[3] = {(tr - t0.x) * hx, (typ.y - tym.y) * hy, (tzp.y - tzm.y) * hz};
                    const float bv[3] = {(rr - r0.x) * hx, (ryp.y - rym.y) * hy, (rzp.y - rzm.y) * hz};
                    const float psi = ngf_residual(av, bv, a.tau, a.rho, vb);
                    if (out)
                        psi_sum.add(psi);
                }
            }
            if (rowB) {
                float *vq = sm + OFF_V + (zB & 3) * 3 * PLANE + sp;
                sts2(vq, va[0], vb[0]);
                sts2(vq + PLANE, va[1], vb[1]);
                sts2(vq + 2 * PLANE, va[2], vb[2]);
            }
        }
        // ---- C: r on plane zA - 4 (rows 2 .. 29), x reduction into node columns
        const int zC = zA - 4;
        if (rowC && zC >= z0 && zC < zend) {   // uniform per warp (a warp holds rows 2w, 2w + 1)
            float ra[3] = {0.f, 0.f, 0.f}, rb[3] = {0.f, 0.f, 0.f};
            // v_x of the pair and of its x neighbours (columns 2tx - 1, 2tx + 2) from the threads beside it
            const float *V0 = sm + OFF_V + (zC & 3) * 3 * PLANE + sp;
            const float2 vx = lds2(V0);
            const float vl = __shfl_up_sync(0xffffffffu, vx.y, 1, BX), vr = __shfl_down_sync(0xffffffffu, vx.x, 1, BX);
            if (outxy && col_in && zC < mz) {
                const float *Vzm = sm + OFF_V + ((zC - 1) & 3) * 3 * PLANE + 2 * PLANE + sp;
                const float *Vzp = sm + OFF_V + ((zC + 1) & 3) * 3 * PLANE + 2 * PLANE + sp;
                const float2 vyp = lds2(V0 + PLANE + CW), vym = lds2(V0 + PLANE - CW);
                const float2 vzm = lds2(Vzm), vzp = lds2(Vzp);
                const float gja = half_hbar * ((vl - vx.y) * hx + (vym.x - vyp.x) * hy + (vzm.x - vzp.x) * hz);
                const float gjb = half_hbar * ((vx.x - vr) * hx + (vym.y - vyp.y) * hy + (vzm.y - vzp.y) * hz);
                const float *gq = sm + OFF_G + (zC & 7) * 3 * PLANE + sp;
                const float2 g0 = lds2(gq), g1 = lds2(gq + PLANE), g2 = lds2(gq + 2 * PLANE);
                ra[0] = gja * g0.x;
                ra[1] = gja * g1.x;
                ra[2] = gja * g2.x;
                rb[0] = gjb * g0.y;
                rb[1] = gjb * g1.y;
                rb[2] = gjb * g2.y;
            }
            // node column j (0..14) gathers columns 2j .. 2j+3 with weights 1/4, 3/4,
            // 3/4, 1/4: the first two are thread j's pair, the last two thread j+1's
            float *red = sm + OFF_RED + (ODD ? 0 : 1) * RED_PLANE + ty * NX * 3;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float lo = 0.25f * ra[c] + 0.75f * rb[c], hi = 0.75f * ra[c] + 0.25f * rb[c];
                const float nv = lo + __shfl_down_sync(0xffffffffu, hi, 1, BX);
                if (tx < NX)
                    red[tx * 3 + c] = nv;
            }
        }
        // ---- D: y reduction of plane zA - 5 (written last step) and accumulation
        // along z: an even plane gives 3/4 to the lower node plane of its interval
        // and 1/4 to the upper, an odd plane the reverse
        const int zD = zA - 5;
        if (zD >= z0 && zD < zend) {
            const float *red = sm + OFF_RED + (ODD ? 1 : 0) * RED_PLANE;
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
        cp_async_wait_all();
        __syncthreads();
    };

    // prologue: node planes of the first interval, then the loads of plane z0 - 2
    {
        const int K0 = (z0 - 2) >> 1;
        issue_node_plane(nc, a.ub, a.dir, sm, K0, g.n[2], node_plane);
        issue_node_plane(nc, a.ub, a.dir, sm, K0 + 1, g.n[2], node_plane);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        a_issue(z0 - 2, std::false_type{}, true);
        cp_async_wait_all();
        __syncthreads();
    }

    // z0 is even: zA + 1 is odd on even steps
    const int nsteps = tz + 7;
    for (int s = 0; s < nsteps; s += 2) {
        step(s, std::true_type{});
        if (s + 1 < nsteps)
            step(s + 1, std::false_type{});
    }
    double ssum = block_sum_to_f64(psi_sum.s, reinterpret_cast<double *>(sm + OFF_RED));
    if (tid == 0)
        a.partials[tile_lin] = ssum;
}

template <bool HAS_DIR, typename IMG = float>
__global__ void __launch_bounds__(BX * BY, 1) k_ngf_fused(FusedArgs a)
{
    extern __shared__ float sm[];
    fused_tile<HAS_DIR, IMG>(a, blockIdx.x, sm);
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
        fused_tile<HAS_DIR, IMG>(a, item - __ldg(tile_off + p), sm);
        __syncthreads();   // the next tile reuses the shared rings
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
// alpha hbar_y L^T w (curvature), one thread per node, 3 components.
// Along x and y the node's owner tile column is t = min(k / 14, nt - 1) at
// local index j = k - 14 t; when j = 0 and t > 0 the lower column also holds
// it, at j = 14.  Along z its owner is the segment holding its node plane
// (node_seg); at the segment's first plane the previous segment also holds it,
// at its last plane.  The up to 8 partials are added owner first, lower x
// before lower y before lower z.
__device__ __forceinline__ void gather_grad_body(const LevelGeom &g, const float *__restrict__ part,
                                                 const FusedSplit &sp, int ntx, int nty,
                                                 const float *__restrict__ w, float alpha_hy,
                                                 float *__restrict__ grad, int bx, int by, int bz)
{
    const int kx = bx * blockDim.x + threadIdx.x;
    const int ky = by * blockDim.y + threadIdx.y;
    const int kz = bz;
    if (kx >= g.n[0] || ky >= g.n[1])
        return;   // (only this function: a caller's barrier after it is still reached)
    const int tx = min(kx / (NX - 1), ntx - 1), ty = min(ky / (NY - 1), nty - 1);
    const int jx = kx - (NX - 1) * tx, jy = ky - (NY - 1) * ty;
    int so, jz;
    node_seg(sp, kz, so, jz);
    const bool lx = jx == 0 && tx > 0, ly = jy == 0 && ty > 0, lz = jz == 0 && so > 0;
    const long long ncols = (long long)ntx * nty, col = tx + (long long)ntx * ty;
    int z0, len;
    sp.seg(so, z0, len);
    const long long stride_o = (long long)(len / 2 + 1) * NE;   // one tile column of the owner segment
    const float *po = part + sp.planes_before(so) * ncols * NE + col * stride_o + (jz * NE + jy * NX + jx);
    long long stride_l = stride_o;
    const float *pl = po;
    if (lz) {   // the previous segment's last node plane
        sp.seg(so - 1, z0, len);
        stride_l = (long long)(len / 2 + 1) * NE;
        pl = part + sp.planes_before(so - 1) * ncols * NE + col * stride_l + ((len / 2) * NE + jy * NX + jx);
    }
    float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const bool ux = q & 1, uy = (q >> 1) & 1, uz = q >> 2;
        if ((ux && !lx) || (uy && !ly) || (uz && !lz))
            continue;
        const long long stride = uz ? stride_l : stride_o;
        // the lower column's copy: one column back, local index 14 instead of 0
        const float *p = (uz ? pl : po) + (ux ? -stride + (NX - 1) : 0) + (uy ? -stride * ntx + (NY - 1) * NX : 0);
        s[0] += __ldg(p);
        s[1] += __ldg(p + NX * NY);
        s[2] += __ldg(p + 2 * NX * NY);
    }
    const int n0 = g.n[0], n01 = g.n[0] * g.n[1];
    const int k = kx + n0 * ky + n01 * kz;
    const int st[3] = {1, n0, n01};
    const int j[3] = {kx, ky, kz};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float *wc = w + c * g.nn;
        const float w0 = __ldg(wc + k);
        float l = 0.f;
#pragma unroll
        for (int e = 0; e < 3; e++) {
            const float lo = j[e] > 0 ? __ldg(wc + k - st[e]) : 0.f;
            const float hi = j[e] < g.n[e] - 1 ? __ldg(wc + k + st[e]) : 0.f;
            l = fmaf(lo + hi - 2.f * w0, g.iH2[e], l);
        }
        grad[c * g.nn + k] = fmaf(alpha_hy, l, s[c]);
    }
}

__global__ void __launch_bounds__(256) k_gather_grad(LevelGeom g, const float *__restrict__ part, FusedSplit sp,
                                                     int ntx, int nty, const float *__restrict__ w, float alpha_hy,
                                                     float *__restrict__ grad)
{
    gather_grad_body(g, part, sp, ntx, nty, w, alpha_hy, grad, blockIdx.x, blockIdx.y, blockIdx.z);
}

// The end of an evaluation in the gather launch.  The final reduction reads
// only the D and S block partials of the kernels before, not the gradient, so
// block 0 reduces them into scal = [J, D, S] (the fixed order of
// finalize_body) and, for phase >= 0, takes that L-BFGS control phase (the
// Armijo decision of a trial point) first, while the other blocks gather.
struct FinArgs {
    const double *pD, *pS;  // block partials of D (fused tiles) and S (curvature blocks)
    int nD, nS;
    double hbar_half, alpha, hy_half;
    double *scal;
    int phase;              // -1: no control phase
    LbfgsState *st;
    unsigned long long h_ls;
};

__global__ void __launch_bounds__(256) k_gather_fin(LevelGeom g, const float *__restrict__ part, FusedSplit sp,
                                                    int ntx, int nty, const float *__restrict__ w, float alpha_hy,
                                                    float *__restrict__ grad, FinArgs f)
{
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
        finalize_body(f.pD, f.nD, f.pS, f.nS, f.hbar_half, f.alpha, f.hy_half, f.scal);
        if (f.phase >= 0) {
            __syncthreads();
            lb_control_body(f.phase, f.st, nullptr, 0, f.scal, f.h_ls, 0ULL, 0ULL);
        }
    }
    gather_grad_body(g, part, sp, ntx, nty, w, alpha_hy, grad, blockIdx.x, blockIdx.y, blockIdx.z);
}

}  // namespace

bool fused_eligible(const Level &L)
{
    for (int d = 0; d < 3; d++)
        if ((L.m[d] & 1) || L.n[d] != L.m[d] / 2 + 1)
            return false;
    return true;
}

// z segment lengths the throughput rule picks from (even: a segment covers
// whole node intervals)
constexpr int TZ_CAND[] = {2, 4, 8, 16, 32, 64, 128};

// Pipeline steps a segment pays beyond its planes (fill and drain)
constexpr int FUSED_FILL = 7;
// longest z segment cfg.fused_tz may force
constexpr int TZ_MAX = 512;

static int fused_cols(const int m[3]) { return ((m[0] + OX - 1) / OX) * ((m[1] + OY - 1) / OY); }

FusedSplit fused_split_uniform(int tz, int mz)
{
    FusedSplit sp;
    sp.l1 = tz;
    sp.n1 = mz / tz;
    sp.lr = mz - sp.n1 * tz;   // even, as mz and tz are
    return sp;
}

// Even z segment lengths that cut a depth of mz planes into ntz = 1, 2, ...
// nearly equal segments, tz = 2 ceil(mz / (2 ntz)), longest first, each once.
static std::vector<int> tz_splits(int mz)
{
    std::vector<int> v;
    for (int ntz = 1;; ntz++) {
        const int tz = 2 * ((mz + 2 * ntz - 1) / (2 * ntz));
        if (tz <= TZ_MAX && (v.empty() || tz < v.back()))
            v.push_back(tz);
        if (tz <= 2)
            break;
    }
    return v;
}

// Load model of the pass.  A tile costs its planes + 7 steps, times a weight
// for the share of its 32 x 32 columns inside the image (columns outside skip
// the loads, the interpolation and the NGF work; about a third of a step's
// work remains).  One CTA is resident per SM and the next free SM takes the
// next tile in launch order (tile_seg_col), so the model replays that order
// and returns the time the last SM finishes.
struct SplitModel {
    std::vector<double> colw;   // weight of each tile column, in column order
    int mz, sms;
    SplitModel(const int m[3], int num_sms) : mz(m[2]), sms(num_sms > 0 ? num_sms : 1)
    {
        const int ntx = (m[0] + OX - 1) / OX, nty = (m[1] + OY - 1) / OY;
        auto frac = [](int t, int o, int width, int extent) {
            int n = 0;
            for (int i = t * o - 2; i < t * o - 2 + width; i++)
                n += i >= 0 && i < extent;
            return (double)n / width;
        };
        for (int ty = 0; ty < nty; ty++)
            for (int tx = 0; tx < ntx; tx++)
                colw.push_back(0.35 + 0.65 * frac(tx, OX, CW, m[0]) * frac(ty, OY, BY, m[1]));
    }
    double makespan(const FusedSplit &sp) const
    {
        // segment groups by length, longest first (stable), as tile_seg_col
        int len[3] = {sp.l1, sp.l2, sp.lr}, cnt[3] = {sp.n1, sp.n2, sp.lr > 0 ? 1 : 0};
        int ord[3] = {0, 1, 2};
        std::stable_sort(ord, ord + 3, [&](int x, int y) { return len[x] > len[y]; });
        std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
        for (int i = 0; i < sms; i++)
            free_at.push(0.0);
        double end = 0.0;
        for (int k = 0; k < 3; k++)
            for (int seg = 0; seg < cnt[ord[k]]; seg++)
                for (double w : colw) {
                    const double t = free_at.top() + w * (len[ord[k]] + FUSED_FILL);
                    free_at.pop();
                    free_at.push(t);
                    end = std::max(end, t);
                }
        return end;
    }
};

// Candidate splits of a depth: the equal splits, and for depths of 32 planes
// and more one or two segments of l1 planes, one to three of l2 < l1 and the
// remainder (lengths on a grid of mz / 32 planes).
static std::vector<FusedSplit> split_candidates(int mz)
{
    std::vector<FusedSplit> v;
    for (int tz : tz_splits(mz))
        v.push_back(fused_split_uniform(tz, mz));
    if (mz >= 32) {
        const int step = std::max(2, (mz / 32) & ~1);
        for (int l1 = step; l1 <= mz; l1 += step)
            for (int n1 = 1; n1 <= 2 && n1 * l1 <= mz; n1++)
                for (int l2 = step; l2 < l1; l2 += step)
                    for (int n2 = 1; n2 <= 3 && n1 * l1 + n2 * l2 <= mz; n2++) {
                        FusedSplit sp;
                        sp.l1 = l1;
                        sp.n1 = n1;
                        sp.l2 = l2;
                        sp.n2 = n2;
                        sp.lr = mz - n1 * l1 - n2 * l2;
                        v.push_back(sp);
                    }
    }
    return v;
}

// candidate splits, cheapest first under the load model (ties: fewer segments)
static std::vector<FusedSplit> splits_ranked(const int m[3], int num_sms)
{
    const SplitModel model(m, num_sms);
    std::vector<std::pair<double, FusedSplit>> r;
    for (const FusedSplit &sp : split_candidates(m[2]))
        r.push_back({model.makespan(sp), sp});
    std::stable_sort(r.begin(), r.end(), [](const std::pair<double, FusedSplit> &x,
                                            const std::pair<double, FusedSplit> &y) {
        if (x.first != y.first)
            return x.first < y.first;
        return x.second.count() < y.second.count();
    });
    std::vector<FusedSplit> v;
    for (auto &e : r)
        v.push_back(e.second);
    return v;
}

FusedSplit fused_split(const Level &L, int num_sms) { return L.split.valid() ? L.split : splits_ranked(L.m, num_sms)[0]; }

FusedSplit fused_split_plan(const int m[3], int num_sms, double *model_steps)
{
    const FusedSplit sp = splits_ranked(m, num_sms)[0];
    if (model_steps)
        *model_steps = SplitModel(m, num_sms).makespan(sp);
    return sp;
}

// Throughput rule: the z segment length of TZ_CAND with the fewest pipeline
// steps in total, ntz * (tz + 7) (ties: the longer one).  The right choice
// when other work keeps every SM busy (a batch of pairs); a single pair alone
// wants segments that fill the GPU in whole waves, which the load model and
// the autotuner find.
int fused_tz_throughput(const Level &L)
{
    int best = 0;
    long long best_steps = 0;
    for (int tz : TZ_CAND) {
        const long long steps = (long long)((L.m[2] + tz - 1) / tz) * (tz + FUSED_FILL);
        if (best == 0 || steps <= best_steps) {
            best = tz;
            best_steps = steps;
        }
    }
    return best;
}

bool fused_tz_valid(int tz) { return tz >= 2 && tz <= TZ_MAX && tz % 2 == 0; }

// tile-partial floats of the level, for any split: a tile of a segment of len
// planes keeps len / 2 + 1 node planes, and the segments' lengths add up to
// the depth, so a split keeps at most depth / 2 + count <= depth planes per column
size_t fused_part_floats(const Level &L, int num_sms)
{
    (void)num_sms;
    return (size_t)fused_cols(L.m) * (size_t)(L.m[2] + 2) * NE;
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
    a.split = fused_split(L, c->num_sms);
    a.ntx = (L.m[0] + OX - 1) / OX;
    a.nty = (L.m[1] + OY - 1) / OY;
    a.part = c->es.part;
    a.partials = partials;
    const int ntiles = a.ntx * a.nty * a.split.count();
    dim3 blk(BX, BY, 1), grd(ntiles, 1, 1);
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
    *n_partials = ntiles;
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_gather_fin(reg_ctx *c, int level, const float *w, float alpha_hy, float *grad, int nD,
                              const double *pS, int nS, double *scal, int phase, cudaStream_t s)
{
    const Level &L = c->L[level];
    const FusedSplit sp = fused_split(L, c->num_sms);
    const int ntx = (L.m[0] + OX - 1) / OX, nty = (L.m[1] + OY - 1) / OY;
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
    f.phase = phase;
    f.st = c->lb.st;
    f.h_ls = phase >= 0 ? lbfgs_graph_handle_ls() : 0ULL;
    k_gather_fin<<<gn, blk, 0, s>>>(L.geom(), c->es.part, sp, ntx, nty, w, alpha_hy, grad, f);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_gather_grad(reg_ctx *c, int level, const float *w, float alpha_hy, float *grad, cudaStream_t s)
{
    const Level &L = c->L[level];
    const FusedSplit sp = fused_split(L, c->num_sms);
    const int ntx = (L.m[0] + OX - 1) / OX, nty = (L.m[1] + OY - 1) / OY;
    dim3 blk(32, 8, 1);
    dim3 gn((L.n[0] + 31) / 32, (L.n[1] + 7) / 8, L.n[2]);
    k_gather_grad<<<gn, blk, 0, s>>>(L.geom(), c->es.part, sp, ntx, nty, w, alpha_hy, grad);
    c->launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Autotuner of the z segmentation of the fused pass.  The candidates are the
// TUNE_CAND splits the load model ranks cheapest plus its two best equal
// splits (in case the model misjudges the weights); for each the pass runs on
// the level's own images at u = u_zero (one warm launch, then the median of
// three CUDA-event timings) and the fastest wins.  Short segments start more
// CTAs (small levels fill the GPU) but pay the 7 pipeline-fill steps and the
// shared node planes more often, and the last CTAs may leave SMs idle, so the
// best split depends on the level and the GPU.  Choices are cached per (image
// dims, SM count, image type, device) for the life of the process: handles of
// the same geometry tune once and pick the same tiling.
// ---------------------------------------------------------------------------
namespace {
constexpr int TUNE_CAND = 6;
std::mutex g_tune_mu;
std::map<std::array<int, 6>, FusedSplit> g_tune;
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
            L.split = it->second;
            return cudaSuccess;
        }
    }
    const std::vector<FusedSplit> ranked = splits_ranked(L.m, c->num_sms);
    std::vector<FusedSplit> cand;
    for (const FusedSplit &sp : ranked)
        if ((int)cand.size() < TUNE_CAND)
            cand.push_back(sp);
    int uniform = 0;
    for (const FusedSplit &sp : ranked) {
        if (uniform == 2)
            break;
        if (sp.n2 == 0 && (sp.lr == 0 || sp.n1 == 0)) {   // equal segments (no remainder)
            uniform++;
            if (std::find(cand.begin(), cand.end(), sp) == cand.end())
                cand.push_back(sp);
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    FusedSplit best;
    float best_ms = 0.f;
    for (const FusedSplit &sp : cand) {
        if (e != cudaSuccess)
            break;
        L.split = sp;
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
        if (!best.valid() || med < best_ms) {
            best = sp;
            best_ms = med;
        }
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        L.split = FusedSplit();
        return e;
    }
    L.split = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Explicit-buffer launches of the fused pass and its gather, for callers that
// own every buffer themselves (the allocation-free entry point).  Geometry
// comes in as a LevelGeom of a ratio-2 grid; no per-dimension tables are used.
// The split is the load model's first choice for the dims (cached per dims).
// ---------------------------------------------------------------------------
static FusedSplit fused_split_dims(const int m[3], int num_sms)
{
    static std::mutex mu;
    static std::map<std::array<int, 4>, FusedSplit> cache;
    const std::array<int, 4> key{m[0], m[1], m[2], num_sms};
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end())
        return it->second;
    const FusedSplit sp = splits_ranked(m, num_sms)[0];
    cache[key] = sp;
    return sp;
}

void fused_layout_dims(const int m[3], int num_sms, int *tz, int *tiles, size_t *part_floats)
{
    const FusedSplit sp = fused_split_dims(m, num_sms);
    const int ncols = fused_cols(m);
    *tz = sp.longest();
    *tiles = ncols * sp.count();
    *part_floats = (size_t)ncols * sp.planes_before(sp.count()) * NE;
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
    a.split = fused_split_dims(g.m, num_sms);
    a.ntx = (g.m[0] + OX - 1) / OX;
    a.nty = (g.m[1] + OY - 1) / OY;
    a.part = part;
    a.partials = partials;
    dim3 blk(BX, BY, 1), grd(a.ntx * a.nty * a.split.count(), 1, 1);
    k_ngf_fused<false><<<grd, blk, SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gather_grad_raw(const LevelGeom &g, const float *part, int num_sms, const float *w,
                                   float alpha_hy, float *grad, cudaStream_t s)
{
    const FusedSplit sp = fused_split_dims(g.m, num_sms);
    const int ntx = (g.m[0] + OX - 1) / OX, nty = (g.m[1] + OY - 1) / OY;
    dim3 blk(32, 8, 1);
    dim3 gn((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, g.n[2]);
    k_gather_grad<<<gn, blk, 0, s>>>(g, part, sp, ntx, nty, w, alpha_hy, grad);
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
        gather_grad_body(P.geom, a.part, a.split, a.ntx, a.nty, P.w, P.alpha_hy, mode ? P.gt : P.g, bx,
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
void fused_tiling(const Level &L, int num_sms, FusedSplit *split, int *ntx, int *nty)
{
    *split = fused_split(L, num_sms);
    *ntx = (L.m[0] + OX - 1) / OX;
    *nty = (L.m[1] + OY - 1) / OY;
}
