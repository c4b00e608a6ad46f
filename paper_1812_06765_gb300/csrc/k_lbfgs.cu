// Device-resident L-BFGS with Armijo backtracking (Sec. 2.1: L-BFGS of Nocedal
// 1980 inside the multilevel scheme).
//
// The direction p = -H g is formed with the compact representation of the
// L-BFGS matrix (Byrd, Nocedal and Schnabel 1994), which equals the two-loop
// recursion in exact arithmetic but needs only two passes over the history:
// one multi-dot pass (fused with the accept step) and one combination pass.
// All scalar decisions (coefficients, curvature test, Armijo test, stopping)
// are taken in FP64 on the device (lbfgs_control.cuh) by the block that
// completes the cross-block reduction of the kernel before them, so the host
// never has to read a scalar to continue, and an iteration can be replayed as
// one CUDA graph.
//
// Vectors (n = 3 * nodes floats): u, g (accepted), gt (trial gradient),
// pdir (current direction), P and Y rings of m + 1 slots each (s_j = t_j P_j).
#include <math.h>

#include <algorithm>
#include <atomic>

#include "batch.h"
#include "fused_pass.cuh"
#include "internal.h"
#include "lbfgs_control.cuh"

namespace {

constexpr int VT = LB_VT;           // threads of the vector kernels

// Reduce ND per-thread values over the block; entry `imax` (if >= 0) by max,
// the others by sum, in FP32 and a fixed order (warp shuffles, then the warp
// totals by one thread per entry); write the block totals to out[0 .. ND) for
// the cross-block double-float sum.
template <int ND>
__device__ __forceinline__ void block_reduce_write(float (&v)[ND], int imax, float *out)
{
    __shared__ float sm[VT / 32][ND];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < ND; d++) {
        float x = (d == imax) ? warp_max(v[d]) : warp_sum(v[d]);
        if (lane == 0)
            sm[warp][d] = x;
    }
    __syncthreads();
    if (threadIdx.x < ND) {
        int d = threadIdx.x;
        float s = sm[0][d];
        for (int w = 1; w < VT / 32; w++)
            s = (d == imax) ? fmaxf(s, sm[w][d]) : s + sm[w][d];
        out[d] = s;
    }
}

// Called by every block of a vector pass after block_reduce_write (see VecTail).
// The arrivals follow the pattern of a grid barrier: block barrier, one
// thread's fence, atomic; the last block's thread fences again before the
// block reads the others' partials.  preloaded: ctl_state() holds the state.
__device__ __forceinline__ void vec_tail(const VecTail &t, const float *__restrict__ partials, int nd, int imax,
                                         int bx, int nblocks, bool preloaded = false)
{
    __shared__ int s_last;
    if (nblocks <= LB_DIRECT) {
        if (t.phase < 0)
            return;   // the control kernel that follows reduces the block partials
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_acq_rel_gpu();   // this block's partials, before its arrival is counted
            s_last = atomicAdd(&t.cnt[0], 1u) == (unsigned)(nblocks - 1);
            if (s_last) {
                fence_acq_rel_gpu();   // every block's partials, before they are read
                t.cnt[0] = 0;
            }
        }
        __syncthreads();
        if (!s_last)
            return;
        lb_control_body(t.phase, t.st, partials, nullptr, nblocks, t.scal, t.h_ls, t.h_iter, t.h_redo, preloaded);
        return;
    }
    __syncthreads();
    const int g = bx / LB_RG, g0 = g * LB_RG, gs = min(LB_RG, nblocks - g0);
    const int ng = (nblocks + LB_RG - 1) / LB_RG;
    if (threadIdx.x == 0) {
        fence_acq_rel_gpu();
        s_last = atomicAdd(&t.cnt[g], 1u) == (unsigned)(gs - 1);
        if (s_last)
            fence_acq_rel_gpu();
    }
    __syncthreads();
    if (!s_last)
        return;
    for (int d = threadIdx.x; d < nd; d += blockDim.x) {   // the max entry: a max of absolute values
        const DFloat x = df_ordered_reduce(partials, (long long)g0 * nd + d, gs, nd, d == imax);
        t.gpart[(size_t)g * nd + d] = make_float2(x.hi, x.lo);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        t.cnt[g] = 0;
        fence_acq_rel_gpu();
        s_last = atomicAdd(&t.cnt[ng], 1u) == (unsigned)(ng - 1);
        if (s_last) {
            fence_acq_rel_gpu();
            t.cnt[ng] = 0;
        }
    }
    __syncthreads();
    if (!s_last || t.phase < 0)
        return;
    lb_control_body(t.phase, t.st, nullptr, t.gpart, ng, t.scal, t.h_ls, t.h_iter, t.h_redo, preloaded);
}

// All vector passes read and write 16-byte vectors: u, g, gt and pdir are
// separate allocations and the P / Y ring slots sit at a stride that is a
// multiple of 4 floats.  The n % 4 tail is done by the first threads of block 0.
__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ float max4(float4 a)
{
    return fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w)));
}

__device__ __forceinline__ void lb_init_dots_body(long long n, const float *__restrict__ g,
                                                     float *__restrict__ partials, const VecTail &tail, int bx,
                                                     int gdx)
{
    float v[2] = {0.f, 0.f};
    const long long n4 = n >> 2;
    const float4 *g4 = reinterpret_cast<const float4 *>(g);
    for (long long e = bx * (long long)VT + threadIdx.x; e < n4; e += (long long)gdx * VT) {
        float4 x = g4[e];
        v[0] += dot4(x, x);
        v[1] = fmaxf(v[1], max4(x));
    }
    if (bx == 0 && threadIdx.x < (n & 3)) {
        float x = g[4 * n4 + threadIdx.x];
        v[0] = fmaf(x, x, v[0]);
        v[1] = fmaxf(v[1], fabsf(x));
    }
    block_reduce_write<2>(v, 1, partials + 2 * bx);
    vec_tail(tail, partials, 2, 1, bx, gdx);
}

__global__ void __launch_bounds__(VT) k_lb_init_dots(long long n, const float *__restrict__ g,
                                                     float *__restrict__ partials, VecTail tail)
{
    lb_init_dots_body(n, g, partials, tail, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Bulk streaming of the direction and accept passes.  Each reads 1 + 2 m or
// 4 + 2 m vectors of n floats and is bound by HBM.  Loads issued by threads
// kept about half the HBM bandwidth busy at 16 warps per SM, whether the
// bytes in flight came from more warps or from more loads per thread, so the
// passes stream their inputs instead with bulk asynchronous copies
// (cp.async.bulk, the TMA engine) into a ring of shared-memory stages.  Each
// stage completes on its own mbarrier, and the threads compute from shared
// memory.  A block owns the chunks bx, bx + gdx, ... of CHUNK4 float4 per
// vector (thread t takes float4 t of each); thread 0 keeps every stage in
// flight.
// ---------------------------------------------------------------------------
constexpr int CHUNK4 = VT;                       // float4 per vector and chunk: one per thread
constexpr int CHUNK_BYTES = CHUNK4 * 16;         // 4 KB
constexpr int VEC_SMEM = 200 * 1024;             // dynamic shared memory of a vector-pass block
constexpr int MAX_STAGES = 4;
constexpr unsigned long long WAIT_NS = 1000000000ULL;   // a stage barrier not complete after 1 s: the pass gives up

// stages that fit for NS vectors per chunk
constexpr int stages_for(int ns)
{
    return VEC_SMEM / (ns * CHUNK_BYTES) < MAX_STAGES ? VEC_SMEM / (ns * CHUNK_BYTES) : MAX_STAGES;
}

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long *b)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
// bytes (a multiple of 16, both addresses 16-byte aligned) from global to shared, completing on b
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *b)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(b))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity)
{
    unsigned done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(smem_addr(b)), "r"(parity)
                 : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// true once the barrier's phase of this parity has completed; false once WAIT_NS have passed
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity)
{
    if (mbar_try_wait(b, parity))
        return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(b, parity))
            return true;
        if (global_ns() - t0 > WAIT_NS)
            return false;
    }
}

// The stage ring of one vector pass: STAGES stages of NS vectors x CHUNK4 float4.
template <int NS>
struct ChunkRing {
    static constexpr int STAGES = stages_for(NS);
    static_assert(STAGES >= 2, "a chunk of every vector must fit twice");
    float4 *buf;                      // dynamic shared memory, VEC_SMEM bytes
    unsigned long long *full;         // [MAX_STAGES] barriers, static shared memory
    long long n4, first;              // float4 per vector; this block's first chunk
    int gdx, chunks;                  // chunk stride; chunks of this block
    bool reverse;                     // walk the block's chunks from its last to its first

    __device__ ChunkRing(float4 *b, unsigned long long *f, long long n4_, int bx, int gdx_, bool reverse_ = false)
        : buf(b), full(f), n4(n4_), first(bx), gdx(gdx_), reverse(reverse_)
    {
        const long long nch = (n4 + CHUNK4 - 1) / CHUNK4;
        chunks = nch > bx ? (int)((nch - 1 - bx) / gdx + 1) : 0;
        if (threadIdx.x == 0) {
            for (int i = 0; i < STAGES; i++)
                mbar_init(&full[i], 1);
            mbar_fence_init();
        }
        __syncthreads();
    }
    __device__ long long elem0(int k) const
    {
        return (first + (long long)(reverse ? chunks - 1 - k : k) * gdx) * CHUNK4;
    }
    __device__ float4 *stage(int k) const { return buf + (size_t)(k % STAGES) * NS * CHUNK4; }
    // thread 0: copy chunk k of the NS source vectors src(i) into its stage;
    // drop (test hook): arm the stage's barrier but issue no copy
    template <typename Src>
    __device__ void issue(int k, Src src, bool drop = false) const
    {
        const long long e0 = elem0(k);
        const long long left = n4 - e0;
        const unsigned bytes = (unsigned)((left < CHUNK4 ? left : CHUNK4) * 16);
        unsigned long long *b = &full[k % STAGES];
        float4 *dst = stage(k);
        mbar_expect_tx(b, bytes * NS);
        if (drop)
            return;
#pragma unroll
        for (int i = 0; i < NS; i++)
            bulk_g2s(dst + i * CHUNK4, src(i) + e0, bytes, b);
    }
    __device__ bool wait(int k) const { return mbar_wait(&full[k % STAGES], (unsigned)((k / STAGES) & 1)); }
    // after a failed wait at chunk k: wait (bounded) for the copies still in flight, chunks k .. k + STAGES - 1
    __device__ void drain(int k) const
    {
        for (int j = k; j < chunks && j < k + STAGES; j++)
            (void)wait(j);
    }
    __device__ void release() const
    {
        __syncthreads();
        if (threadIdx.x == 0)
            for (int i = 0; i < STAGES; i++)
                mbar_inval(&full[i]);
        __syncthreads();
    }
};

// Streams the chunks of a block through the ring: compute(k, stage) per chunk.
// Returns false if a stage never completed (the block's sums are then
// incomplete and the caller flags the pass).  drop_first: test hook, the
// first chunk's copies are not issued.
template <int NS, typename Src, typename Compute>
__device__ __forceinline__ bool stream_chunks(ChunkRing<NS> &ring, Src src, Compute compute, bool drop_first = false)
{
    constexpr int S = ChunkRing<NS>::STAGES;
    if (threadIdx.x == 0)
        for (int k = 0; k < S && k < ring.chunks; k++)
            ring.issue(k, src, drop_first && k == 0);
    for (int k = 0; k < ring.chunks; k++) {
        const bool ok = ring.wait(k);
        if (ok)
            compute(k, ring.stage(k));
        // every thread is done with the stage (or one timed out: all leave together)
        if (!__syncthreads_and(ok)) {
            ring.drain(k);
            ring.release();
            return false;
        }
        if (threadIdx.x == 0 && k + S < ring.chunks)
            ring.issue(k + S, src);
    }
    ring.release();
    return true;
}

// direction for DC stored pairs from one stage: vectors g, P_0..P_{DC-1}, Y_0..Y_{DC-1}
template <int DC>
__device__ __forceinline__ bool direction_stream(long long n4, int bx, int gdx, float cg, const float4 *g4,
                                                 const float4 *P4, const float4 *Y4, const int (&off)[LB_MAXM],
                                                 const float (&cp)[LB_MAXM], const float (&cy)[LB_MAXM],
                                                 float4 *__restrict__ p4, float (&v)[2], float4 *buf,
                                                 unsigned long long *full, bool drop_first)
{
    constexpr int NS = 1 + 2 * DC;
    // the reverse of the accept pass's order: the chunks that pass read last
    // (the history's high ends) are still in L2 when this pass starts
    ChunkRing<NS> ring(buf, full, n4, bx, gdx, true);
    auto src = [&](int i) -> const float4 * { return i == 0 ? g4 : (i <= DC ? P4 + off[i - 1] : Y4 + off[i - 1 - DC]); };
    return stream_chunks<NS>(ring, src, [&](int k, const float4 *sb) {
        const long long e = ring.elem0(k) + threadIdx.x;
        if (e >= n4)
            return;
        const float4 gv = sb[threadIdx.x];
        float4 p = make_float4(cg * gv.x, cg * gv.y, cg * gv.z, cg * gv.w);
#pragma unroll
        for (int j = 0; j < DC; j++) {
            const float4 a = sb[(1 + j) * CHUNK4 + threadIdx.x], b = sb[(1 + DC + j) * CHUNK4 + threadIdx.x];
            p.x = fmaf(cp[j], a.x, fmaf(cy[j], b.x, p.x));
            p.y = fmaf(cp[j], a.y, fmaf(cy[j], b.y, p.y));
            p.z = fmaf(cp[j], a.z, fmaf(cy[j], b.z, p.z));
            p.w = fmaf(cp[j], a.w, fmaf(cy[j], b.w, p.w));
        }
        p4[e] = p;
        v[0] += dot4(gv, p);
        v[1] += dot4(p, p);
    }, drop_first);
}

// p = cg g + sum_j cp_j P_j + cy_j Y_j, written to pdir; partial sums of g'p and p'p.
__device__ __forceinline__ void lb_direction_body(long long n, long long stride, const LbfgsState *st,
                                                     const float *__restrict__ g, const float *__restrict__ P,
                                                     const float *__restrict__ Y, float *__restrict__ pdir,
                                                     float *__restrict__ partials, int redo, const VecTail &tail,
                                                     int bx, int gdx)
{
    __shared__ int s_run, s_dc, s_slot[LB_MAXM];
    __shared__ float s_cg, s_cp[LB_MAXM], s_cy[LB_MAXM];
    ctl_state_load(st);   // also the copy the control phase works on
    __syncthreads();
    if (threadIdx.x == 0) {
        const LbfgsState &S = ctl_state();
        s_run = redo ? S.redo_dir : (S.iter_continue && !S.done);
        s_dc = S.dcount;
        s_cg = (float)S.cg;
        for (int j = 0; j < LB_MAXM; j++) {
            s_slot[j] = S.dslot[j];
            s_cp[j] = (float)S.cp[j];
            s_cy[j] = (float)S.cy[j];
        }
    }
    __syncthreads();
    if (!s_run && tail.phase < 0)   // nothing to compute and no control phase to reach: done
        return;
    float v[2] = {0.f, 0.f};
    if (s_run) {   // otherwise only the arrival below (partials unused)
        const int dc = s_dc;
        const float cg = s_cg;
        // slot j of both rings starts off[j] float4s in (the slot stride is a multiple of 4 floats)
        const float4 *P4 = reinterpret_cast<const float4 *>(P), *Y4 = reinterpret_cast<const float4 *>(Y);
        int off[LB_MAXM];
        float cp[LB_MAXM], cy[LB_MAXM];
#pragma unroll
        for (int j = 0; j < LB_MAXM; j++) {
            off[j] = j < dc ? (int)(s_slot[j] * (stride >> 2)) : 0;
            cp[j] = s_cp[j];
            cy[j] = s_cy[j];
        }
        const long long n4 = n >> 2;
        const float4 *g4 = reinterpret_cast<const float4 *>(g);
        float4 *p4 = reinterpret_cast<float4 *>(pdir);
        extern __shared__ float4 vec_buf[];
        __shared__ unsigned long long s_full[MAX_STAGES];
        const bool drop = bx == 0 && ctl_state().test_drop;   // test hook: one chunk goes missing
        bool ok;
        switch (dc) {
        case 0: ok = direction_stream<0>(n4, bx, gdx, cg, g4, P4, Y4, off, cp, cy, p4, v, vec_buf, s_full, drop); break;
        case 1: ok = direction_stream<1>(n4, bx, gdx, cg, g4, P4, Y4, off, cp, cy, p4, v, vec_buf, s_full, drop); break;
        case 2: ok = direction_stream<2>(n4, bx, gdx, cg, g4, P4, Y4, off, cp, cy, p4, v, vec_buf, s_full, drop); break;
        case 3: ok = direction_stream<3>(n4, bx, gdx, cg, g4, P4, Y4, off, cp, cy, p4, v, vec_buf, s_full, drop); break;
        case 4: ok = direction_stream<4>(n4, bx, gdx, cg, g4, P4, Y4, off, cp, cy, p4, v, vec_buf, s_full, drop); break;
        case 5: ok = direction_stream<5>(n4, bx, gdx, cg, g4, P4, Y4, off, cp, cy, p4, v, vec_buf, s_full, drop); break;
        case 6: ok = direction_stream<6>(n4, bx, gdx, cg, g4, P4, Y4, off, cp, cy, p4, v, vec_buf, s_full, drop); break;
        case 7: ok = direction_stream<7>(n4, bx, gdx, cg, g4, P4, Y4, off, cp, cy, p4, v, vec_buf, s_full, drop); break;
        default: ok = direction_stream<8>(n4, bx, gdx, cg, g4, P4, Y4, off, cp, cy, p4, v, vec_buf, s_full, drop); break;
        }
        if (!ok && threadIdx.x == 0)
            atomicOr(const_cast<int *>(&st->wait_err), 1);
        if (bx == 0 && threadIdx.x < (n & 3)) {
            const long long e = 4 * n4 + threadIdx.x;
            float gv = __ldcg(g + e), p = cg * gv;
#pragma unroll
            for (int j = 0; j < LB_MAXM; j++)
                if (j < dc)
                    p = fmaf(cp[j], __ldcg(P + (size_t)s_slot[j] * stride + e),
                             fmaf(cy[j], __ldcg(Y + (size_t)s_slot[j] * stride + e), p));
            pdir[e] = p;
            v[0] = fmaf(gv, p, v[0]);
            v[1] = fmaf(p, p, v[1]);
        }
    }
    block_reduce_write<2>(v, -1, partials + 2 * bx);
    vec_tail(tail, partials, 2, -1, bx, gdx, true);
}

__global__ void __launch_bounds__(VT) k_lb_direction(long long n, long long stride, const LbfgsState *st,
                                                     const float *__restrict__ g, const float *__restrict__ P,
                                                     const float *__restrict__ Y, float *__restrict__ pdir,
                                                     float *__restrict__ partials, int redo, VecTail tail)
{
    lb_direction_body(n, stride, st, g, P, Y, pdir, partials, redo, tail, blockIdx.x, gridDim.x);
}

// Accept the trial point: u += t pdir (the fmaf the evaluation used), store the
// candidate pair in the free slot (P = pdir, Y = g_new - g), g = g_new, and
// take every dot the next direction needs in the same pass: with g_new and with
// y_new against every stored P and Y (the free slot, always the last list
// entry, from registers), plus g_new'g_new and ||g_new||_inf.
__device__ __forceinline__ void accept_elem(float gn, float go, float pf, float &u, float t, float &yn)
{
    yn = gn - go;
    u = fmaf(t, pf, u);
}

// accept for NP stored pairs before the free slot from one stage: vectors
// g_new, g, p, u, P_0..P_{NP-1}, Y_0..Y_{NP-1}; the stored slots are never the
// free slot this pass writes
template <int NP>
__device__ __forceinline__ bool accept_stream(long long n4, int bx, int gdx, float t, const float4 *gt4, float4 *g4,
                                              const float4 *pd4, float4 *u4, const float4 *P4, const float4 *Y4,
                                              const int (&off)[LB_MAXM], float4 *Pf4, float4 *Yf4,
                                              float (&v)[ND_ACC], float (&fr)[4], float4 *buf,
                                              unsigned long long *full)
{
    constexpr int NS = 4 + 2 * NP;
    ChunkRing<NS> ring(buf, full, n4, bx, gdx);
    auto src = [&](int i) -> const float4 * {
        return i == 0 ? gt4 : i == 1 ? g4 : i == 2 ? pd4 : i == 3 ? u4 : (i < 4 + NP ? P4 + off[i - 4] : Y4 + off[i - 4 - NP]);
    };
    return stream_chunks<NS>(ring, src, [&](int k, const float4 *sb) {
        const long long e = ring.elem0(k) + threadIdx.x;
        if (e >= n4)
            return;
        const int q = threadIdx.x;
        const float4 gn = sb[q], go = sb[CHUNK4 + q], pf = sb[2 * CHUNK4 + q];
        float4 uu = sb[3 * CHUNK4 + q];
        float4 yn;
        accept_elem(gn.x, go.x, pf.x, uu.x, t, yn.x);
        accept_elem(gn.y, go.y, pf.y, uu.y, t, yn.y);
        accept_elem(gn.z, go.z, pf.z, uu.z, t, yn.z);
        accept_elem(gn.w, go.w, pf.w, uu.w, t, yn.w);
        v[0] += dot4(gn, gn);
        v[1] = fmaxf(v[1], max4(gn));
#pragma unroll
        for (int j = 0; j < NP; j++) {
            const float4 pj = sb[(4 + j) * CHUNK4 + q], yj = sb[(4 + NP + j) * CHUNK4 + q];
            v[2 + 4 * j] += dot4(pj, gn);
            v[3 + 4 * j] += dot4(yj, gn);
            v[4 + 4 * j] += dot4(pj, yn);
            v[5 + 4 * j] += dot4(yj, yn);
        }
        fr[0] += dot4(pf, gn);
        fr[1] += dot4(yn, gn);
        fr[2] += dot4(pf, yn);
        fr[3] += dot4(yn, yn);
        u4[e] = uu;
        g4[e] = gn;
        Pf4[e] = pf;
        Yf4[e] = yn;
    });
}

__device__ __forceinline__ void lb_accept_body(long long n, long long stride, const LbfgsState *st,
                                                  float *__restrict__ u, float *__restrict__ g,
                                                  const float *__restrict__ gt, const float *__restrict__ pdir,
                                                  float *__restrict__ P, float *__restrict__ Y,
                                                  float *__restrict__ partials, const VecTail &tail, int bx,
                                                  int gdx)
{
    __shared__ int s_ok, s_lc, s_free, s_slot[LB_MAXS];
    __shared__ float s_t;
    ctl_state_load(st);   // also the copy the control phase works on
    __syncthreads();
    if (threadIdx.x == 0) {
        const LbfgsState &S = ctl_state();
        s_ok = S.active && S.ls == LS_ACCEPTED;
        s_lc = S.lcount;
        s_free = S.free_slot;
        s_t = (float)S.t;
        for (int j = 0; j < LB_MAXS; j++)
            s_slot[j] = S.lslot[j];
    }
    __syncthreads();
    if (!s_ok && tail.phase < 0)   // nothing to compute and no control phase to reach: done
        return;
    float v[ND_ACC];
#pragma unroll
    for (int d = 0; d < ND_ACC; d++)
        v[d] = 0.f;
    if (s_ok) {   // otherwise only the arrival below (partials unused)
        const int np = s_lc - 1;    // stored pairs before the free slot
        const float t = s_t;
        const float4 *P4 = reinterpret_cast<const float4 *>(P), *Y4 = reinterpret_cast<const float4 *>(Y);
        int off[LB_MAXM];   // slot j of both rings starts off[j] float4s in
#pragma unroll
        for (int j = 0; j < LB_MAXM; j++)
            off[j] = j < np ? (int)(s_slot[j] * (stride >> 2)) : 0;
        float *Pf = P + (size_t)s_free * stride;
        float *Yf = Y + (size_t)s_free * stride;
        float fr[4] = {0.f, 0.f, 0.f, 0.f};   // dots of the free slot (p, y_new) with g_new, y_new
        const long long n4 = n >> 2;
        const float4 *gt4 = reinterpret_cast<const float4 *>(gt), *pd4 = reinterpret_cast<const float4 *>(pdir);
        float4 *g4 = reinterpret_cast<float4 *>(g), *u4 = reinterpret_cast<float4 *>(u);
        float4 *Pf4 = reinterpret_cast<float4 *>(Pf), *Yf4 = reinterpret_cast<float4 *>(Yf);
        extern __shared__ float4 vec_buf[];
        __shared__ unsigned long long s_full[MAX_STAGES];
        bool ok;
#define ACCEPT_CASE(K) ok = accept_stream<K>(n4, bx, gdx, t, gt4, g4, pd4, u4, P4, Y4, off, Pf4, Yf4, v, fr, vec_buf, s_full)
        switch (np) {
        case 0: ACCEPT_CASE(0); break;
        case 1: ACCEPT_CASE(1); break;
        case 2: ACCEPT_CASE(2); break;
        case 3: ACCEPT_CASE(3); break;
        case 4: ACCEPT_CASE(4); break;
        case 5: ACCEPT_CASE(5); break;
        case 6: ACCEPT_CASE(6); break;
        case 7: ACCEPT_CASE(7); break;
        default: ACCEPT_CASE(8); break;
        }
#undef ACCEPT_CASE
        if (!ok && threadIdx.x == 0)
            atomicOr(const_cast<int *>(&st->wait_err), 1);
        if (bx == 0 && threadIdx.x < (n & 3)) {
            const long long e = 4 * n4 + threadIdx.x;
            float gn = __ldcg(gt + e), go = __ldcg(g + e), pf = __ldcg(pdir + e), uu = __ldcg(u + e), yn;
            accept_elem(gn, go, pf, uu, t, yn);
            u[e] = uu;
            g[e] = gn;
            Pf[e] = pf;
            Yf[e] = yn;
            v[0] = fmaf(gn, gn, v[0]);
            v[1] = fmaxf(v[1], fabsf(gn));
#pragma unroll
            for (int j = 0; j < LB_MAXM; j++)
                if (j < np) {   // unrolled with a predicate so that v stays in registers
                    float pj = __ldcg(P + (size_t)s_slot[j] * stride + e), yj = __ldcg(Y + (size_t)s_slot[j] * stride + e);
                    v[2 + 4 * j] = fmaf(pj, gn, v[2 + 4 * j]);
                    v[3 + 4 * j] = fmaf(yj, gn, v[3 + 4 * j]);
                    v[4 + 4 * j] = fmaf(pj, yn, v[4 + 4 * j]);
                    v[5 + 4 * j] = fmaf(yj, yn, v[5 + 4 * j]);
                }
            fr[0] = fmaf(pf, gn, fr[0]);
            fr[1] = fmaf(yn, gn, fr[1]);
            fr[2] = fmaf(pf, yn, fr[2]);
            fr[3] = fmaf(yn, yn, fr[3]);
        }
        // the free slot is list position np
#pragma unroll
        for (int j = 0; j < LB_MAXS; j++)
            if (j == np) {
                v[2 + 4 * j] += fr[0];
                v[3 + 4 * j] += fr[1];
                v[4 + 4 * j] += fr[2];
                v[5 + 4 * j] += fr[3];
            }
    }
    block_reduce_write<ND_ACC>(v, 1, partials + (size_t)ND_ACC * bx);
    vec_tail(tail, partials, ND_ACC, 1, bx, gdx, true);
}

__global__ void __launch_bounds__(VT) k_lb_accept(long long n, long long stride, const LbfgsState *st,
                                                  float *__restrict__ u, float *__restrict__ g,
                                                  const float *__restrict__ gt, const float *__restrict__ pdir,
                                                  float *__restrict__ P, float *__restrict__ Y,
                                                  float *__restrict__ partials, VecTail tail)
{
    lb_accept_body(n, stride, st, u, g, gt, pdir, P, Y, partials, tail, blockIdx.x, gridDim.x);
}

// Reduction of an objective evaluation's block partials (J, D, S into scal)
// followed, in the same block, by a control phase on those scalars (ARMIJO
// after a trial evaluation).
__global__ void __launch_bounds__(512) k_finalize_ctl(const double *__restrict__ pD, int nD,
                                                      const double *__restrict__ pS, int nS, double hbar_half,
                                                      double alpha, double hy_half, double *scal, int phase,
                                                      LbfgsState *st, unsigned long long h_ls,
                                                      unsigned long long h_iter)
{
    finalize_body(pD, nD, pS, nS, hbar_half, alpha, hy_half, scal);
    __syncthreads();
    lb_control_body(phase, st, nullptr, nullptr, 0, scal, h_ls, h_iter, 0ULL);
}

// ---------------------------------------------------------------------------
// Batched forms: one launch covers the vectors (or the states) of all pairs.
// A vector item is (pair, block) and runs the per-pair body with that pair's
// block count, so every pair gets exactly the partial sums it gets alone.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(VT) k_lb_vector_batch(const PairLevel *__restrict__ pl,
                                                        const int *__restrict__ chunk_off, int npairs, int total,
                                                        int step)
{
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int p = find_pair(chunk_off, npairs, item);
        const PairLevel &P = pl[p];
        const int b = item - __ldg(chunk_off + p);
        const VecTail tail{P.lgpart, P.lcnt, -1, P.st, nullptr, 0ULL, 0ULL, 0ULL};   // control: its own kernel
        if (step == 0)
            lb_init_dots_body(P.n, P.g, P.lpart, tail, b, P.nchunks);
        else if (step == 1 || step == 2)
            lb_direction_body(P.n, P.stride, P.st, P.g, P.P, P.Y, P.pdir, P.lpart, step == 2, tail, b, P.nchunks);
        else
            lb_accept_body(P.n, P.stride, P.st, P.u, P.g, P.gt, P.pdir, P.P, P.Y, P.lpart, tail, b, P.nchunks);
        __syncthreads();   // the next item reuses the block's shared staging
    }
}

// one block per pair: control phase `phase` of each pair, on its group sums; scalars of the objective at u
// (INIT) or at the trial point (ARMIJO)
__global__ void __launch_bounds__(CT) k_lb_control_batch(const PairLevel *__restrict__ pl, int phase)
{
    const PairLevel &P = pl[blockIdx.x];
    const bool direct = P.nchunks <= LB_DIRECT;   // block partials, else group sums (vec_tail)
    lb_control_body(phase, P.st, direct ? P.lpart : nullptr, direct ? nullptr : P.lgpart,
                    direct ? P.nchunks : (P.nchunks + LB_RG - 1) / LB_RG,
                    phase == LB_INIT ? P.scal : P.scal_t, 0ULL, 0ULL, 0ULL);
}

// condition of a batched loop: 1 while any pair still iterates (which = 0) or
// still searches (which = 1)
__global__ void k_batch_condition(const PairLevel *__restrict__ pl, int npairs, int which, unsigned long long h,
                                  int *__restrict__ counters)
{
    if (threadIdx.x == 0 && counters)
        counters[which]++;   // counters[2 + which]: the last value (read by a host-driven loop)
    int any = 0;
    for (int p = threadIdx.x; p < npairs; p += 32) {
        const LbfgsState *st = pl[p].st;
        any |= which == 0 ? st->iter_continue : (st->active && st->ls_continue);
    }
    any = __any_sync(0xffffffffu, any);
    if (threadIdx.x == 0 && counters)
        counters[2 + which] = any;
#if CUDART_VERSION >= 12040
    if (threadIdx.x == 0 && h)
        cudaGraphSetConditional((cudaGraphConditionalHandle)h, any ? 1u : 0u);
#endif
}

// Standalone direction for a given set of pairs (reg_lbfgs_direction): the
// dots of S, Y and g one at a time (entry 0: g'g, 1: ||g||_inf, then S_i'g,
// Y_i'g, then S_i'Y_j, Y_i'Y_j).  Only used by that entry point.
__device__ __forceinline__ void pair_dot_operands(int d, int count, long long n, long long e,
                                                  const float *__restrict__ S, const float *__restrict__ Y,
                                                  const float *__restrict__ g, float &a, float &b)
{
    int q = d - 2;
    if (q < 2 * count) {
        int i = q >> 1;
        a = (q & 1) ? Y[(size_t)i * n + e] : S[(size_t)i * n + e];
        b = g[e];
    } else {
        q -= 2 * count;
        int i = (q >> 1) / count, j = (q >> 1) % count;
        a = (q & 1) ? Y[(size_t)i * n + e] : S[(size_t)i * n + e];
        b = Y[(size_t)j * n + e];
    }
}

__global__ void __launch_bounds__(VT) k_lb_pair_dots(long long n, int count, const float *__restrict__ S,
                                                     const float *__restrict__ Y, const float *__restrict__ g,
                                                     float *__restrict__ partials)
{
    const int nd = 2 + 2 * count + 2 * count * count;
    for (int d = 0; d < nd; d++) {
        float acc = 0.f;
        for (long long e = blockIdx.x * (long long)VT + threadIdx.x; e < n; e += (long long)gridDim.x * VT) {
            if (d == 0) {
                acc = fmaf(g[e], g[e], acc);
            } else if (d == 1) {
                acc = fmaxf(acc, fabsf(g[e]));
            } else {
                float a, b;
                pair_dot_operands(d, count, n, e, S, Y, g, a, b);
                acc = fmaf(a, b, acc);
            }
        }
        float v[1] = {acc};
        __syncthreads();
        block_reduce_write<1>(v, d == 1 ? 0 : -1, partials + (size_t)blockIdx.x * nd + d);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(VT) k_lb_direction_plain(long long n, const LbfgsState *__restrict__ st,
                                                           const float *__restrict__ g, const float *__restrict__ S,
                                                           const float *__restrict__ Y, float *__restrict__ p)
{
    const int dc = st->dcount;
    const float cg = (float)st->cg;
    for (long long e = blockIdx.x * (long long)VT + threadIdx.x; e < n; e += (long long)gridDim.x * VT) {
        float v = cg * g[e];
        for (int j = 0; j < dc; j++) {
            size_t o = (size_t)st->dslot[j] * n + e;
            v = fmaf((float)st->cp[j], S[o], fmaf((float)st->cy[j], Y[o], v));
        }
        p[e] = v;
    }
}

__global__ void k_lb_pair_setup(LbfgsState *__restrict__ st, int count, const float *__restrict__ partials,
                                int nblocks)
{
    const int nd = 2 + 2 * count + 2 * count * count;
    if (threadIdx.x == 0) {
        double red[2 + 2 * LB_MAXM + 2 * LB_MAXM * LB_MAXM];
        for (int d = 0; d < nd; d++) {
            double s = 0.0;
            for (int b = 0; b < nblocks; b++) {
                double x = partials[(size_t)b * nd + d];
                s = (d == 1) ? fmax(s, x) : s + x;
            }
            red[d] = s;
        }
        st->gg = red[0];
        st->ginf = red[1];
        st->count = count;
        for (int i = 0; i < count; i++) {
            st->order[i] = i;
            st->tscale[i] = 1.0;
            st->Pg[i] = red[2 + 2 * i];
            st->Yg[i] = red[3 + 2 * i];
            for (int j = 0; j < count; j++) {
                int q = 2 + 2 * count + 2 * (i * count + j);
                st->SY[i][j] = red[q];
                st->YY[i][j] = red[q + 1];
            }
            st->iSY[i] = 1.0 / st->SY[i][i];
        }
        if (count > 0)
            st->gamma = st->SY[count - 1][count - 1] / st->YY[count - 1][count - 1];
        else
            set_p0(st);
        st->iter_continue = 1;
        st->done = 0;
    }
    __syncwarp();
    if (count > 0)
        set_compact_warp(st);
}

// ---------------------------------------------------------------------------
// Whole-level loop of small levels (Sec. 2.1: L-BFGS with Armijo backtracking
// in the multilevel scheme).  One cooperative launch runs every iteration of
// the level with the level graph's device code: the direction pass, the p0
// redo when its control asks for one, each line-search trial (the fused pass
// at u + t p with the curvature formed in the pass, then the node gather with
// the final reduction and the Armijo decision in block 0) and the accept pass.
// A grid barrier replaces each kernel boundary; the control phases still run
// in the block that completes each cross-block reduction.  On levels of a few
// thousand to a few hundred thousand nodes the kernel boundaries, conditional
// nodes and ramp-ups of the graph cost as much as the work.
// ---------------------------------------------------------------------------
struct LevelLoopArgs {
    FusedArgs fa;               // trial point: ub = u, dir = pdir, t_dev = &st->t
    int ntiles;                 // tiles of the fused pass
    int gather_items, gather_runs;   // gather blocks, and runs per node plane
    float alpha_hy;             // alpha hbar_y of the curvature gradient
    double hbar_half, alpha, hy_half;
    double *scal_t;             // [J, D, S] of the trial point
    long long n, stride;        // vector length, ring slot stride
    float *u, *g, *gt, *pdir, *P, *Y;
    float *partials;            // FP32 block partials of the vector passes
    int nvec;                   // blocks of the vector passes (as the level graph's)
    VecTail tdir, tredo, tacc;  // their folded reductions and control phases
    LbfgsState *st;
    unsigned *bar;              // [arrivals, generation, flag snapshot] of the grid barrier
    int max_steps;              // bound on the loop bodies and trials
};

__device__ __forceinline__ int ld_flag(const int *p) { return *reinterpret_cast<const volatile int *>(p); }

// loop flags of the state, as the block that releases a grid barrier saw them
constexpr unsigned F_ITER = 1u, F_REDO = 2u, F_LS = 4u, F_ERR = 8u;

// Grid-wide barrier of the cooperative launch (every block resident): block
// barrier, one thread's release fence and arrival.  The last block to arrive
// takes a snapshot of the state's loop flags (iteration, p0 redo, line search,
// copy-wait error), resets the count and advances the generation; the others
// wait for it, at most WAIT_NS, and read the snapshot.  Every block so takes
// the loop decisions from the same flags, whatever a control phase writes
// later.  Returns false, and the caller's block leaves the kernel, on an
// error flag or an expired wait (which flags the state: the level stops; the
// other blocks leave at their next barrier).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, LbfgsState *st, unsigned &flags)
{
    __shared__ unsigned s_flags;
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1, *snap = bar + 2;
        const unsigned g0 = *gen;
        int ok = 1;
        fence_acq_rel_gpu();   // this block's writes, before its arrival is counted
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            fence_acq_rel_gpu();   // every block's writes, before the snapshot reads them
            *snap = (ld_flag(&st->iter_continue) ? F_ITER : 0u) | (ld_flag(&st->redo_dir) ? F_REDO : 0u) |
                    (ld_flag(&st->ls_continue) ? F_LS : 0u) | (ld_flag(&st->wait_err) ? F_ERR : 0u);
            bar[0] = 0;
            fence_acq_rel_gpu();   // the snapshot and the reset, before the release
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g0) {
                if (global_ns() - t0 > WAIT_NS) {
                    ok = 0;
                    atomicOr(&st->wait_err, 1);
                    break;
                }
                __nanosleep(100);
            }
        }
        fence_acq_rel_gpu();   // the snapshot and every block's writes, before this block reads them
        s_flags = *snap;
        s_ok = ok && !(s_flags & F_ERR);
    }
    __syncthreads();
    flags = s_flags;
    return s_ok != 0;
}

__global__ void __launch_bounds__(VT, 1) k_level_loop(LevelLoopArgs a)
{
    extern __shared__ float4 dyn4[];
    float *sm = reinterpret_cast<float *>(dyn4);
    const unsigned nb = gridDim.x;
    const int bx = blockIdx.x;
    LbfgsState *st = a.st;
    unsigned f = 0;
    int steps = 0;
    if (!grid_barrier(a.bar, nb, st, f))   // the first snapshot
        return;
    while ((f & F_ITER) && steps++ < a.max_steps) {
        if (bx < a.nvec)
            lb_direction_body(a.n, a.stride, st, a.g, a.P, a.Y, a.pdir, a.partials, 0, a.tdir, bx, a.nvec);
        if (!grid_barrier(a.bar, nb, st, f))
            return;
        if (f & F_REDO) {
            if (bx < a.nvec)
                lb_direction_body(a.n, a.stride, st, a.g, a.P, a.Y, a.pdir, a.partials, 1, a.tredo, bx, a.nvec);
            if (!grid_barrier(a.bar, nb, st, f))
                return;
        }
        while ((f & F_LS) && steps++ < a.max_steps) {
            for (int tile = bx; tile < a.ntiles; tile += nb) {
                fused_tile<true, float, true, true>(a.fa, tile, sm);
                __syncthreads();   // the next tile reuses the shared rings
            }
            if (!grid_barrier(a.bar, nb, st, f))
                return;
            if (bx == 0) {   // J, D, S of the trial point and the Armijo decision, then its gather share
                finalize_body(a.fa.partials, a.ntiles, a.fa.partials_S, a.ntiles, a.hbar_half, a.alpha, a.hy_half,
                              a.scal_t);
                __syncthreads();
                lb_control_body(LB_ARMIJO, st, nullptr, nullptr, 0, a.scal_t, 0ULL, 0ULL, 0ULL);
            }
            for (int item = bx; item < a.gather_items; item += nb)
                gather_grad_body<true>(a.fa.g, a.fa.part, a.fa.split, a.fa.ntx, a.fa.nty, a.fa.w, a.alpha_hy, a.gt,
                                       item % a.gather_runs, item / a.gather_runs);
            if (!grid_barrier(a.bar, nb, st, f))
                return;
        }
        if (bx < a.nvec)
            lb_accept_body(a.n, a.stride, st, a.u, a.g, a.gt, a.pdir, a.P, a.Y, a.partials, a.tacc, bx, a.nvec);
        if (!grid_barrier(a.bar, nb, st, f))
            return;
    }
    if (steps > a.max_steps && bx == 0 && threadIdx.x == 0) {   // cannot happen with the control's own bounds
        st->status = -6;
        st->done = 1;
        st->iter_continue = 0;
    }
}

}  // namespace

// Blocks of the vector passes that fit on one SM at once (the fewer of the
// accept and direction kernels, whose register counts set it; at most 4, the
// group buffers' bound).  With every block resident the grid-stride loops run
// in one wave instead of a full wave and a partial one.
// The streamed vector passes take VEC_SMEM bytes of dynamic shared memory,
// above the 48 KB default: the limit is raised once per device (before the
// first launch, which may be inside a stream capture).
cudaError_t lbfgs_kernels_setup(int device)
{
    static std::atomic<bool> done[64];
    const int dev = device >= 0 && device < 64 ? device : 0;
    if (done[dev].load())
        return cudaSuccess;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_lb_direction, at, VEC_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_lb_accept, at, VEC_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_lb_vector_batch, at, VEC_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_level_loop, at, VEC_SMEM);
    if (e == cudaSuccess)
        done[dev].store(true);
    return e;
}

static int vec_blocks_per_sm()
{
    static std::atomic<int> cached{0};
    int v = cached.load();
    if (v > 0)
        return v;
    int a = 0, d = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_lb_accept, VT, VEC_SMEM) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, k_lb_direction, VT, VEC_SMEM) != cudaSuccess) {
        (void)cudaGetLastError();
        return 2;
    }
    v = std::max(1, std::min(4, std::min(a, d)));
    cached.store(v);
    return v;
}

int num_blocks_for(reg_ctx *c, long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    long long cap = (long long)vec_blocks_per_sm() * c->num_sms;
    if (b > cap)
        b = cap;
    if (b < 1)
        b = 1;
    return (int)b;
}

void lbfgs_state_reset_host(LbfgsState *st, const reg_config &cfg, int max_iter, double Hmin)
{
    memset(st, 0, sizeof(*st));
    st->m = cfg.lbfgs_mem;
    st->max_iter = max_iter;
    st->max_bt = cfg.max_backtracks;
    st->fixed_iters = cfg.fixed_iters;
    st->tol_j_count = cfg.tol_j_count;
    st->c1 = cfg.c1;
    st->tol_grad_rel = cfg.tol_grad_rel;
    st->tol_j_rel = cfg.tol_j_rel;
    st->Hmin = Hmin;
    st->t = 1.0;
    st->test_drop = cfg.test_expire_wait;
}

static unsigned long long g_h_ls = 0, g_h_iter = 0, g_h_redo = 0;  // conditional handles while capturing

void lbfgs_set_graph_handles(unsigned long long h_ls, unsigned long long h_iter, unsigned long long h_redo)
{
    g_h_ls = h_ls;
    g_h_iter = h_iter;
    g_h_redo = h_redo;
}

unsigned long long lbfgs_graph_handle_ls() { return g_h_ls; }

// folded reduction + control of a vector pass (handles: the graph conditions
// the phase sets while a level graph is captured)
static VecTail tail_of(reg_ctx *c, int phase, const double *scal, bool use_ls_handle, bool use_iter_handle,
                       bool use_redo_handle = false)
{
    return VecTail{c->lb.gpart, c->lb.cnt, phase, c->lb.st, scal, use_ls_handle ? g_h_ls : 0ULL,
                   use_iter_handle ? g_h_iter : 0ULL, use_redo_handle ? g_h_redo : 0ULL};
}

// ring slots start on 16-byte boundaries
static long long ring_stride(long long n) { return (n + 3) & ~3LL; }

cudaError_t lbfgs_launch_init(reg_ctx *c, int level, cudaStream_t s)
{
    long long n = 3 * c->L[level].nn;
    int nb = num_blocks_for(c, (n + 3) / 4, VT);
    // arrival counters start the level at zero (every launch leaves them so)
    cudaError_t e = cudaMemsetAsync(c->lb.cnt, 0, sizeof(unsigned) * c->lb.cnt_len, s);
    if (e == cudaSuccess)
        e = launch_eval(c, level, c->lb.u, nullptr, nullptr, c->lb.g, c->es.scal, -1, s);
    if (e != cudaSuccess)
        return e;
    k_lb_init_dots<<<nb, VT, 0, s>>>(n, c->lb.g, c->lb.partials, tail_of(c, LB_INIT, c->es.scal, false, true));
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t lbfgs_launch_direction(reg_ctx *c, int level, cudaStream_t s)
{
    long long n = 3 * c->L[level].nn, sd = ring_stride(n);
    int nb = num_blocks_for(c, (n + 3) / 4, VT);
    k_lb_direction<<<nb, VT, VEC_SMEM, s>>>(n, sd, c->lb.st, c->lb.g, c->lb.P, c->lb.Y, c->lb.pdir, c->lb.partials, 0,
                                     tail_of(c, LB_DIR, nullptr, true, false, true));
    c->launches += 1;
    return cudaGetLastError();
}

// the p0 redo: a direction pass that runs only when the compact-form direction
// was not a descent direction (a no-op pass otherwise; a graph runs it under an
// IF node that the direction's control sets)
cudaError_t lbfgs_launch_redo(reg_ctx *c, int level, cudaStream_t s)
{
    long long n = 3 * c->L[level].nn, sd = ring_stride(n);
    int nb = num_blocks_for(c, (n + 3) / 4, VT);
    k_lb_direction<<<nb, VT, VEC_SMEM, s>>>(n, sd, c->lb.st, c->lb.g, c->lb.P, c->lb.Y, c->lb.pdir, c->lb.partials, 1,
                                     tail_of(c, LB_DIR_REDO, nullptr, true, false));
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t lbfgs_launch_direction_level(reg_ctx *c, int level, cudaStream_t s)
{
    cudaError_t e = lbfgs_launch_direction(c, level, s);
    return e == cudaSuccess ? lbfgs_launch_redo(c, level, s) : e;
}

cudaError_t lbfgs_launch_trial(reg_ctx *c, int level, cudaStream_t s)
{
    // the trial point u + t pdir is formed inside the evaluation kernels; the
    // Armijo decision runs in the evaluation's final reduction
    return launch_eval(c, level, c->lb.u, c->lb.pdir, &c->lb.st->t, c->lb.gt, c->lb.scal_t, LB_ARMIJO, s);
}

cudaError_t lbfgs_launch_accept_level(reg_ctx *c, int level, cudaStream_t s)
{
    long long n = 3 * c->L[level].nn, sd = ring_stride(n);
    int nb = num_blocks_for(c, (n + 3) / 4, VT);
    k_lb_accept<<<nb, VT, VEC_SMEM, s>>>(n, sd, c->lb.st, c->lb.u, c->lb.g, c->lb.gt, c->lb.pdir, c->lb.P, c->lb.Y,
                                  c->lb.partials, tail_of(c, LB_ACCEPTED, nullptr, false, true));
    c->launches += 1;
    return cudaGetLastError();
}

// Blocks of the whole-level kernel (all resident at once), 0 where the device
// has no cooperative launch.  Cached per device.
static int level_loop_grid(reg_ctx *c)
{
    static std::atomic<int> cached[64];
    const int dev = c->device >= 0 && c->device < 64 ? c->device : 0;
    int v = cached[dev].load();
    if (v != 0)
        return v > 0 ? v : 0;
    int coop = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
        lbfgs_kernels_setup(c->device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level_loop, VT, VEC_SMEM) != cudaSuccess) {
        (void)cudaGetLastError();
        per_sm = 0;
    }
    v = per_sm > 0 ? per_sm * c->num_sms : -1;
    cached[dev].store(v);
    return v > 0 ? v : 0;
}

bool lbfgs_level_loop_ok(reg_ctx *c, int level)
{
    if (!c->cfg.use_graph || !use_fused(c, level) || !small_level(c, level) || c->cfg.image_dtype != 0)
        return false;
    const int grid = level_loop_grid(c);
    return grid > 0 && num_blocks_for(c, (3 * c->L[level].nn + 3) / 4, VT) <= grid;
}

cudaError_t lbfgs_launch_level_loop(reg_ctx *c, int level, cudaStream_t s)
{
    const Level &L = c->L[level];
    LevelLoopArgs a;
    a.fa = fused_args(c, level, c->lb.u, c->lb.pdir, &c->lb.st->t, c->es.partials, &a.ntiles);
    a.gather_runs = gather_runs_per_plane(L.n);
    a.gather_items = a.gather_runs * L.n[2];
    const double hy = L.H[0] * L.H[1] * L.H[2];
    a.alpha_hy = (float)(c->cfg.alpha * hy);
    a.hbar_half = 0.5 * L.h[0] * L.h[1] * L.h[2];
    a.alpha = c->cfg.alpha;
    a.hy_half = 0.5 * hy;
    a.scal_t = c->lb.scal_t;
    a.n = 3 * L.nn;
    a.stride = ring_stride(a.n);
    a.u = c->lb.u;
    a.g = c->lb.g;
    a.gt = c->lb.gt;
    a.pdir = c->lb.pdir;
    a.P = c->lb.P;
    a.Y = c->lb.Y;
    a.partials = c->lb.partials;
    a.nvec = num_blocks_for(c, (a.n + 3) / 4, VT);
    a.tdir = tail_of(c, LB_DIR, nullptr, false, false);
    a.tredo = tail_of(c, LB_DIR_REDO, nullptr, false, false);
    a.tacc = tail_of(c, LB_ACCEPTED, nullptr, false, false);
    a.st = c->lb.st;
    a.bar = c->lb.gbar;
    a.max_steps = 4 * (c->cfg.max_iter[level] + 1) * (c->cfg.max_backtracks + 1) + 16;
    // a launch that ended at an expired barrier may have left arrivals behind
    cudaError_t e = cudaMemsetAsync(c->lb.gbar, 0, 3 * sizeof(unsigned), s);
    if (e != cudaSuccess)
        return e;
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_level_loop), dim3(level_loop_grid(c)),
                                    dim3(VT), args, VEC_SMEM, s);
    c->launches += 1;
    return e;
}

// evaluation reduction with a control phase (k_curv.cu calls this for trial points)
cudaError_t launch_finalize_ctl(reg_ctx *c, const double *pD, int nD, const double *pS, int nS, double hbar_half,
                                double alpha, double hy_half, double *scal, int phase, cudaStream_t s)
{
    k_finalize_ctl<<<1, 512, 0, s>>>(pD, nD, pS, nS, hbar_half, alpha, hy_half, scal, phase, c->lb.st,
                                      phase == LB_ARMIJO ? g_h_ls : 0ULL, 0ULL);
    return cudaGetLastError();
}

cudaError_t lbfgs_direction_standalone(reg_ctx *c, long long n, int count, const float *S, const float *Y,
                                       const float *g, float *p, double Hmin, cudaStream_t s)
{
    int nb = num_blocks_for(c, n, VT);
    k_lb_pair_dots<<<nb, VT, 0, s>>>(n, count, S, Y, g, c->lb.partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    k_lb_pair_setup<<<1, 32, 0, s>>>(c->lb.st, count, c->lb.partials, nb);
    // pairs live in the caller's S, Y: slots 0..count-1 at stride n (any alignment)
    k_lb_direction_plain<<<nb, VT, 0, s>>>(n, c->lb.st, g, S, Y, p);
    c->launches += 3;
    return cudaGetLastError();
}

// batched launchers (batch.cu): step 0 norms of g, 1 direction, 2 its p0 redo, 3 accept
cudaError_t launch_lb_vector_batch(const PairLevel *pl, const int *chunk_off, int npairs, int total, int step,
                                   int grid, cudaStream_t s)
{
    k_lb_vector_batch<<<grid, VT, VEC_SMEM, s>>>(pl, chunk_off, npairs, total, step);
    return cudaGetLastError();
}

cudaError_t launch_lb_control_batch(const PairLevel *pl, int npairs, int phase, cudaStream_t s)
{
    k_lb_control_batch<<<npairs, CT, 0, s>>>(pl, phase);
    return cudaGetLastError();
}

cudaError_t launch_batch_condition(const PairLevel *pl, int npairs, int which, unsigned long long h, int *counters,
                                   cudaStream_t s)
{
    k_batch_condition<<<1, 32, 0, s>>>(pl, npairs, which, h, counters);
    return cudaGetLastError();
}
