// One pyramid level of L-BFGS as one CUDA graph launch.
//
//   init: objective at u0; ||g||, ||g||_inf + control(INIT)      -> sets the iteration condition
//   WHILE (iteration condition)
//       direction + control(DIR)                                    -> sets the redo and line-search conditions
//       IF (redo condition): p0 direction + control(DIR_REDO)
//       WHILE (line-search condition)
//           objective at u + t p; its final reduction + control(ARMIJO)
//       accept (no-op unless accepted) + control(ACCEPTED)        -> sets the iteration condition
//
// Each control phase runs in FP64 in the last block of the kernel before it
// (the block that completes that kernel's cross-block reduction), so a level
// runs without a host round trip and without separate control launches.
// Termination does not depend on the host: every search ends after
// max_backtracks trials, and the control phases end the level after max_iter
// accepted steps, a failed search, a non-finite value, or (a bound that should
// never bind) 2 max_iter + 8 loop bodies.
#include <vector>

#include "internal.h"

namespace {

struct CaptureGuard {   // ends a capture that an early return would leave open
    cudaStream_t s;
    bool active = false;
    ~CaptureGuard()
    {
        if (active) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(s, &g);
        }
    }
};

// leaf nodes of the capture so far (copied: the runtime's array is transient)
cudaError_t capture_leaves(cudaStream_t s, std::vector<cudaGraphNode_t> &out)
{
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &nd);
    if (e != cudaSuccess)
        return e;
    out.assign(deps, deps + nd);
    return cudaSuccess;
}

cudaError_t add_cond(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps, cudaGraphConditionalHandle h,
                     cudaGraphConditionalNodeType type, cudaGraphNode_t *node, cudaGraph_t *body)
{
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaError_t e = cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p);
    if (e == cudaSuccess)
        *body = p.conditional.phGraph_out[0];
    return e;
}

cudaError_t add_while(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps, cudaGraphConditionalHandle h,
                      cudaGraphNode_t *node, cudaGraph_t *body)
{
    return add_cond(g, deps, h, cudaGraphCondTypeWhile, node, body);
}

}  // namespace

// Kernel node priorities of one graph (not its conditional bodies): the
// kernel low_func (the curvature Laplacian, which runs beside the NGF pass) at
// the device's lowest stream priority and every other kernel at the highest,
// so that the block scheduler hands out the NGF pass's CTAs (one per SM) first
// and the curvature blocks take the SMs that the NGF pass's last, shorter tiles
// leave idle.  The graph must be instantiated with
// cudaGraphInstantiateFlagUseNodePriority for the priorities to apply.
cudaError_t set_graph_kernel_priorities(cudaGraph_t g, const void *low_func)
{
    int lowest = 0, highest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lowest, &highest);
    size_t n = 0;
    if (e == cudaSuccess)
        e = cudaGraphGetNodes(g, nullptr, &n);
    if (e != cudaSuccess || n == 0)
        return e;
    std::vector<cudaGraphNode_t> nodes(n);
    e = cudaGraphGetNodes(g, nodes.data(), &n);
    for (size_t i = 0; e == cudaSuccess && i < n; i++) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[i], &t);
        if (e != cudaSuccess || t != cudaGraphNodeTypeKernel)
            continue;
        cudaKernelNodeParams kp = {};
        e = cudaGraphKernelNodeGetParams(nodes[i], &kp);
        if (e != cudaSuccess)
            break;
        cudaLaunchAttributeValue v = {};
        v.priority = kp.func == low_func ? lowest : highest;
        e = cudaGraphKernelNodeSetAttribute(nodes[i], cudaLaunchAttributePriority, &v);
    }
    return e;
}

#define GK(call)                                  \
    do {                                          \
        cudaError_t _e = (call);                  \
        if (_e != cudaSuccess) {                  \
            lbfgs_set_graph_handles(0, 0, 0);        \
            c->launches = launches0;              \
            if (G) cudaGraphDestroy(G);           \
            return _e;                            \
        }                                         \
    } while (0)

// Build (once per level and geometry) the executable graph of a whole level.
cudaError_t build_level_graph(reg_ctx *c, int level, cudaGraphExec_t *out)
{
    const long long launches0 = c->launches;   // capture queues nothing: keep the counter
    cudaGraph_t G = nullptr;
    cudaStream_t cs = c->cap_stream;
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    GK(cudaGraphCreate(&G, 0));
    cudaGraphConditionalHandle h_iter, h_ls;
    GK(cudaGraphConditionalHandleCreate(&h_iter, G, 0, cudaGraphCondAssignDefault));

    std::vector<cudaGraphNode_t> leaves;
    {   // init
        CaptureGuard guard{cs};
        GK(cudaStreamBeginCaptureToGraph(cs, G, nullptr, nullptr, 0, mode));
        guard.active = true;
        lbfgs_set_graph_handles(0, h_iter, 0);
        GK(lbfgs_launch_init(c, level, cs));
        GK(capture_leaves(cs, leaves));
        guard.active = false;
        cudaGraph_t g2 = nullptr;
        GK(cudaStreamEndCapture(cs, &g2));
    }
    cudaGraphNode_t w_iter;
    cudaGraph_t body = nullptr;
    GK(add_while(G, leaves, h_iter, &w_iter, &body));
    cudaGraphConditionalHandle h_redo;
    GK(cudaGraphConditionalHandleCreate(&h_ls, body, 0, cudaGraphCondAssignDefault));
    GK(cudaGraphConditionalHandleCreate(&h_redo, body, 0, cudaGraphCondAssignDefault));
    {   // iteration body: the direction, whose control sets the redo and line-search conditions
        CaptureGuard guard{cs};
        GK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, mode));
        guard.active = true;
        lbfgs_set_graph_handles(h_ls, h_iter, h_redo);
        GK(lbfgs_launch_direction(c, level, cs));
        GK(capture_leaves(cs, leaves));
        guard.active = false;
        cudaGraph_t g2 = nullptr;
        GK(cudaStreamEndCapture(cs, &g2));
    }
    cudaGraphNode_t if_redo;
    cudaGraph_t redo_body = nullptr;
    GK(add_cond(body, leaves, h_redo, cudaGraphCondTypeIf, &if_redo, &redo_body));
    {   // IF (not a descent direction): the p0 direction
        CaptureGuard guard{cs};
        GK(cudaStreamBeginCaptureToGraph(cs, redo_body, nullptr, nullptr, 0, mode));
        guard.active = true;
        lbfgs_set_graph_handles(h_ls, h_iter, 0);
        GK(lbfgs_launch_redo(c, level, cs));
        guard.active = false;
        cudaGraph_t g2 = nullptr;
        GK(cudaStreamEndCapture(cs, &g2));
    }
    leaves.assign(1, if_redo);
    cudaGraphNode_t w_ls;
    cudaGraph_t ls_body = nullptr;
    GK(add_while(body, leaves, h_ls, &w_ls, &ls_body));
    {   // line-search body
        CaptureGuard guard{cs};
        GK(cudaStreamBeginCaptureToGraph(cs, ls_body, nullptr, nullptr, 0, mode));
        guard.active = true;
        lbfgs_set_graph_handles(h_ls, h_iter, 0);
        GK(lbfgs_launch_trial(c, level, cs));
        guard.active = false;
        cudaGraph_t g2 = nullptr;
        GK(cudaStreamEndCapture(cs, &g2));
    }
    {   // accept, after the line search
        CaptureGuard guard{cs};
        GK(cudaStreamBeginCaptureToGraph(cs, body, &w_ls, nullptr, 1, mode));
        guard.active = true;
        lbfgs_set_graph_handles(h_ls, h_iter, 0);
        GK(lbfgs_launch_accept_level(c, level, cs));
        guard.active = false;
        cudaGraph_t g2 = nullptr;
        GK(cudaStreamEndCapture(cs, &g2));
    }
    lbfgs_set_graph_handles(0, 0, 0);
    for (cudaGraph_t g : {G, body, redo_body, ls_body})
        GK(set_graph_kernel_priorities(g, curv_w_kernel()));
    GK(cudaGraphInstantiate(out, G, cudaGraphInstantiateFlagUseNodePriority));
    cudaGraphDestroy(G);
    c->launches = launches0;
    return cudaSuccess;
}

// kernels of one objective evaluation at a level (for the launch statistics)
int eval_kernel_count(const reg_ctx *c, int level)
{
    if (use_fused(c, level)) {   // fused pass, curvature, gather (+ the final reduction beside it on large grids)
        const Level &L = c->L[level];
        return (gather_blocks(L.n) < GATHER_SPLIT_BLOCKS ? 3 : 4) - (fused_curv_in_pass(c, level) ? 1 : 0);
    }
    static const int ngf[3] = {4, 3, 10};   // multi-pass NGF kernels per P^T variant
    return ngf[mp_pt_variant(c, level)] + 3;   // + curvature, its gradient, final reduction
}
