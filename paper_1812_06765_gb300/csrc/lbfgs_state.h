// Device-resident L-BFGS state (FP64 scalars).  One instance per handle; on
// the device only the control phases write it (run by one block: the one that
// completes a kernel's cross-block reduction, or a control kernel of the
// batched form); the host writes it only before a level starts.
#pragma once

#define LB_MAXM 8
#define LB_MAXS (LB_MAXM + 1)   // m pairs + one free slot for the next direction
#define LB_VT 256               // threads of the vector passes (up to 4 blocks per SM)

enum LbPhase { LB_INIT = 0, LB_DIR = 1, LB_DIR_REDO = 2, LB_ARMIJO = 3, LB_ACCEPTED = 4 };
enum LbSearch { LS_RUNNING = 0, LS_ACCEPTED = 1, LS_FAILED = 2, LS_RETRY = 3 };

struct LbfgsState {
    // parameters
    int m, max_iter, max_bt, fixed_iters, tol_j_count;
    double c1, tol_grad_rel, tol_j_rel, Hmin;
    // accepted iterate
    double J, D, S, J0, g0norm, ginf;
    double gtol2;      // (tol_grad_rel * ||g0||)^2: the gradient test compares squares
    // trial point
    double Jt, Dt, St;
    double t;          // current step length
    double gtp, pp;    // g'p and p'p of the current direction
    int k;             // accepted iterations
    int trial;         // trial index inside the current search
    int evals;         // objective evaluations on this level
    int small_count;   // consecutive small-J-change iterations
    int bodies;        // iteration bodies run (accepted steps, retries, the final failed search)
    int retried;       // the p0 retry of this iteration has been used
    int redo_dir;      // the direction must be recomputed as p0
    int redos;         // p0 redos on this level (each one extra direction pass)
    int ls;            // LbSearch
    int ls_continue;   // 1 while the line search needs another trial
    int iter_continue; // 1 while the level needs another iteration
    int active;        // this pair runs the current iteration body (set by the direction
                       // control; in a batch, finished pairs skip every later phase)
    int done;
    int status;        // 0, 1 (line search warning), -5 (numeric), -6 (loop bound), -7 (copy wait expired)
    int wait_err;      // set by a vector pass whose bulk-copy wait expired; the next control phase stops the level
    int test_drop;     // test hook (reg_config.test_expire_wait): the next direction pass loses one chunk
    // pair memory: order[0..count-1] are slots oldest..newest, free_slot holds p
    int count, free_slot;
    int order[LB_MAXM];
    double tscale[LB_MAXS];          // s_slot = tscale * P_slot
    double iSY[LB_MAXS];             // 1 / (s'y) of the pair in the slot
    double gamma;                    // s'y / y'y of the newest stored pair
    double SY[LB_MAXS][LB_MAXS];     // s_i' y_j by slot (upper triangle by age)
    double YY[LB_MAXS][LB_MAXS];     // y_i' y_j by slot
    // direction p = cg g + sum_j cp[j] P[dslot[j]] + cy[j] Y[dslot[j]]
    int dcount;
    int dslot[LB_MAXM];
    double cg, cp[LB_MAXM], cy[LB_MAXM];
    // dots of the last accept pass, by list position (0..count-1 active, count = free)
    int lcount;
    int lslot[LB_MAXS];
    double Pg[LB_MAXS], Yg[LB_MAXS], Py[LB_MAXS], Yy[LB_MAXS];
    double gg;
};

// Cross-block reduction of a vector pass and the control step folded into it.
// Each block writes its FP32 partials.  Blocks are grouped LB_RG at a time:
// the last block of a group (completion order) sums the group's partials in
// block order as double-float pairs, and the block that completes the last
// group runs control phase `phase` on the group sums (-1: none, a separate
// control kernel follows).  Grids of at most LB_DIRECT blocks skip the group
// level (one fence, atomic and serial sum fewer on the critical path): every
// block arrives on one counter and the control reduces the block partials
// themselves.  The sums do not depend on the completion order.
#define LB_RG 16
#define LB_DIRECT 256
struct VecTail {
    float2 *gpart;                   // [groups][nd] group sums, double-float (hi, lo)
    unsigned *cnt;                   // [groups + 1] arrival counters, zero between launches
    int phase;
    LbfgsState *st;
    const double *scal;              // [J, D, S] the phase reads (INIT)
    unsigned long long h_ls, h_iter, h_redo; // graph conditions the phase sets (0: none)
};
