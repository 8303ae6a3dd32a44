// qcd_solve_cg_many: even-odd CG solves of several systems -- each with its
// own gauge field, lattice volume, hopping parameter, twisted mass and
// tolerance -- advanced together by ONE persistent kernel launch.
//
// The paper's finite-temperature studies are many independent runs over
// couplings and lattice sizes, a naturally parallel setup (Sec. 1), bounded
// by device memory (Sec. 2).  For small volumes one solve cannot fill the
// GPU: a launch's fixed cost and the latency of each thread's FP64 work set
// the time, not bandwidth.  Here a cooperative grid stays resident for the
// whole solve of every system: source preparation, the CG iterations on
// Mhat^dag Mhat x_e = Mhat^dag b'_e, the FP64 true-residual check, the odd-
// site reconstruction and the full-system residual, with grid-wide barriers
// between the phases instead of kernel launches.
//
// * Blocks are divided among the systems in proportion to their site
//   counts (at least one each).  Reductions are summed per fixed chunk of
//   work items and the chunks in a fixed order, so every sum -- and every
//   result -- is bitwise the same alone and in any batch.
// * Hopping phases use eight threads per site, one hop each (forward and
//   backward of the four directions): the FP64 work of one thread is an
//   eighth of a site's, which is what bounds the latency of a small
//   lattice on GB300 (an FP64 warp instruction occupies a sub-partition's
//   FP64 unit for 64 cycles).  The eight partial spinors are summed with
//   warp shuffles; the spin projection and the lower-spin rebuild are
//   table-driven (sign and lane selections, no branches on the direction).
// * Every barrier wait is bounded by a clock64 budget.  When it runs out the
//   kernel records QCD_ERR_TIMEOUT and every block returns; the call then
//   fails with that status and the context stays usable.
//
// Conventions as in the other kernels (chiral basis, D_hop with (1 - gamma)
// forward and (1 + gamma) backward, A = 1 + i a gamma_5, a = 2 kappa mu,
// antiperiodic t through t_bc).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "qcd_handles.h"
#include "hop_lanes.cuh"

namespace qcd {
namespace {

#define QCD_CHECK_CUDA(expr, what)                        \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return check_cuda(e_, what); \
    } while (0)

constexpr int kManyThreads = 128;
constexpr int kManyMax = 32;

// A half field of FP64 spinors: 12 planes of double2, site-fastest.
struct HV {
    double2 *d;
    int stride;
};

// Coefficients of one hopping phase: out = cy[chi] y + cd[chi] (D in).
struct PhaseCoef {
    double cy[2][2], cd[2][2];
};

enum ManyPhaseCoef : int {
    MC_SRC_B = 0,   // b' = b_e + kappa D_eo t               (cy = 1, cd = kappa)
    MC_SRC_T,       // t = A^-dag D_oe^dag b'               (cy = 0, cd = A^-dag)
    MC_SRC_R,       // rhs = A^dag b' - kappa^2 D_eo^dag t  (cy = A^dag, cd = -kappa^2)
    MC_OP1,         // t = A^-1 D_oe p
    MC_OP2,         // s = A p - kappa^2 D_eo t
    MC_OP3,         // t = A^-dag D_oe^dag s
    MC_OP4,         // q = A^dag s - kappa^2 D_eo^dag t
    MC_RECON,       // x_o = A^-1 b_o + kappa A^-1 D_oe x_e
    MC_FULL,        // M x = A x - kappa D x
    MC_COUNT
};

struct ManySys {
    Geom g;
    const double2 *U;   // FP64 reconstruct-18 links: block (parity*4 + mu), 9 planes each
    int ustride;
    HV be, bo, xe, xo;  // the caller's b and x
    HV bp, rhs, r, p, q, t, s;
    double tw_inv[2][2];    // A^-1 per chirality (source preparation)
    PhaseCoef pc[MC_COUNT];
    double tol2;
    int block0, nblocks;  // this system's blocks
    int chunk0;           // offset of its reduction chunks in each partial slot
};

enum ManyStatus : int { MS_RUNNING = 0, MS_CONVERGED = 1, MS_DONE = 2, MS_BREAKDOWN = 3, MS_MAXITER = 4 };

struct ManySysState {
    double b2, rr, rr_new, pAp, alpha, beta, rr_stop, rr_true, full_r2, full_b2;
    int status, iter_done;
};

struct ManyState {
    ManySysState s[kManyMax];
    int n;
    int iter, maxiter;
    int reliable;          // true-residual passes
    int error;             // QCD_ERR_TIMEOUT when a barrier wait ran out
    unsigned arrive;       // barrier arrivals (zero at launch)
    unsigned gen;          // barrier generation
    int timeout_where;     // phase index of the first timeout
};

// hop_lane8 and reduce_lanes8 (hop_lanes.cuh) compute the hops, eight
// threads per site.
// ---- grid barrier with a finaliser run by the last block to arrive
//
// Reductions are summed per chunk of kManyThreads consecutive work items of
// a system (whichever block processes the chunk writes its partial), and
// the finaliser adds a system's chunks with the whole block in a fixed
// order.  The result therefore depends neither on how many blocks a system
// gets nor on what else is in the batch.

struct Ctx {
    const ManySys *sys;
    ManyState *st;
    double *part;          // [slot][chunk] partials
    const int *block_sys;  // system of each block
    int n, nblk;
    int nchunk;            // chunks per slot (all systems)
    long long budget;      // clock64 cycles a barrier wait may take
};

// Sum of this block's v (thread 0 gets it), fixed order.
__device__ __forceinline__ double block_total(double v)
{
    __shared__ double sm[32];
    double a[1] = {v};
    block_sum<1>(a, sm);
    return a[0];
}

// A system's total of the chunk partials in `slot` (items_per_site work
// items per site); every thread of the block calls it, thread 0 gets it.
__device__ __forceinline__ double chunk_sum(const Ctx &x, int slot, int k, int items_per_site)
{
    const ManySys &S = x.sys[k];
    const int nc = (S.g.h * items_per_site + kManyThreads - 1) / kManyThreads;
    const double *p = x.part + (size_t)slot * x.nchunk + S.chunk0;
    double a = 0.0;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) a += __ldcg(p + c);
    return block_total(a);
}

// A grid-wide barrier.  Before it, each block has written its chunk
// partials for this phase; the last block to arrive runs `fin` with all its
// threads (sums, CG decisions by thread 0), then releases the others.
// Returns false when the wait ran out (the kernel must return).
template <typename Fin>
__device__ bool grid_barrier(const Ctx &x, int where, Fin fin)
{
    __shared__ int ok, last;
    __shared__ unsigned my_gen;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        my_gen = *(volatile unsigned *)&x.st->gen;
        __threadfence();
        last = atomicAdd(&x.st->arrive, 1u) == (unsigned)x.nblk - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        fin();
        __syncthreads();
        if (threadIdx.x == 0) {
            x.st->arrive = 0;
            __threadfence();
            atomicAdd(&x.st->gen, 1u);
        }
    } else if (threadIdx.x == 0) {
        volatile unsigned *genp = &x.st->gen;
        const long long t0 = clock64();
        while (*genp == my_gen) {
            if (*(volatile int *)&x.st->error != 0 || clock64() - t0 > x.budget) {
                if (atomicCAS(&x.st->error, 0, QCD_ERR_TIMEOUT) == 0) x.st->timeout_where = where;
                ok = 0;
                break;
            }
        }
        __threadfence();
    }
    if (threadIdx.x == 0 && *(volatile int *)&x.st->error != 0) ok = 0;
    __syncthreads();
    return ok != 0;
}

// ---- phases

// A hopping phase: for every system, out (parity p) = cy y + cd D in on the
// system's blocks, eight threads per site; optionally |out|^2 -> slot.
// With `full` both parities are done and only |b - out|^2, |b|^2 are
// reduced (slots 0 and 1), nothing is stored.
__device__ void hop_phase(const Ctx &x, int k, int lb, int coef, int p, bool dagger, HV ManySys::*in, HV ManySys::*y,
                          HV ManySys::*out, int red_slot, bool skip_done)
{
    const ManySys &S = x.sys[k];
    const PhaseCoef &pc = S.pc[coef];
    const int run = __ldcg(&x.st->s[k].status);
    if (!(skip_done && run != MS_RUNNING)) {
        const int items = S.g.h * 8;
        for (int base = lb * blockDim.x; base < items; base += S.nblocks * blockDim.x) {
            const int w = base + threadIdx.x;
            const bool act = w < items;
            double red = 0.0;
            const int i = w >> 3, lane = w & 7;
            cx<double> acc[12];
            if (act) {
                hop_lane8<true>(S.g, S.U, S.ustride, (S.*in).d, (S.*in).stride, p, i, lane, dagger, acc);
            } else {
#pragma unroll
                for (int a = 0; a < 12; ++a) acc[a] = mk(0.0, 0.0);
            }
            reduce_lanes8(acc, lane);
            if (act && !(lane & 1)) {
                const int spin = ((lane >> 2) << 1) | ((lane >> 1) & 1), chi = spin >> 1;
                const cx<double> cd = mk(pc.cd[chi][0], pc.cd[chi][1]), cy = mk(pc.cy[chi][0], pc.cy[chi][1]);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int plane = 3 * spin + a;
                    cx<double> v = cmul(cd, acc[a]);
                    if (y) {
                        const double2 yy = __ldcg((S.*y).d + (size_t)plane * (S.*y).stride + i);
                        v = cmac(v, cy, mk(yy.x, yy.y));
                    }
                    if (!out) {
                        // full residual: |b - M x|^2 and |b|^2 (b of this parity)
                        const HV &bh = p == 0 ? S.be : S.bo;
                        const double2 bb = __ldg(bh.d + (size_t)plane * bh.stride + i);
                        const double dr = bb.x - v.re, di = bb.y - v.im;
                        red += dr * dr + di * di;
                    } else {
                        const HV &o = S.*out;
                        o.d[(size_t)plane * o.stride + i] = make_double2(v.re, v.im);
                        if (red_slot >= 0) red += v.re * v.re + v.im * v.im;
                    }
                }
            }
            if (red_slot >= 0) {
                const double t = block_total(red);
                if (threadIdx.x == 0) x.part[(size_t)red_slot * x.nchunk + S.chunk0 + base / blockDim.x] = t;
            }
        }
    }
}

// |b|^2 of a full system (slot), for the full-residual statistics.
__device__ void bnorm_phase(const Ctx &x, int k, int lb, int slot)
{
    const ManySys &S = x.sys[k];
    const int items = S.g.h * 24;  // both parities, 12 complex each
    for (int base = lb * blockDim.x; base < items; base += S.nblocks * blockDim.x) {
        const int w = base + threadIdx.x;
        double red = 0.0;
        if (w < items) {
            const int par = w / (S.g.h * 12), r = w - par * S.g.h * 12, plane = r / S.g.h, i = r - plane * S.g.h;
            const HV &bh = par == 0 ? S.be : S.bo;
            const double2 v = __ldg(bh.d + (size_t)plane * bh.stride + i);
            red = v.x * v.x + v.y * v.y;
        }
        const double t = block_total(red);
        if (threadIdx.x == 0) x.part[(size_t)slot * x.nchunk + S.chunk0 + base / blockDim.x] = t;
    }
}

// Site-local vector phases, one thread per (site, complex component).
enum VecOp : int { V_TWIST_BO, V_SETUP, V_XR, V_P, V_TRUE, V_RESTART };

__device__ void vec_phase(const Ctx &x, int k, int lb, VecOp op, int red_slot)
{
    const ManySys &S = x.sys[k];
    const ManySysState &q = x.st->s[k];
    const int status = __ldcg(&q.status);
    const bool running = status == MS_RUNNING;
    const bool conv = status == MS_CONVERGED;
    bool go = true;
    if (op == V_XR || op == V_P) go = running;
    if (op == V_TRUE || op == V_RESTART) go = conv;
    if (go) {
        const int items = S.g.h * 12;
        for (int base = lb * blockDim.x; base < items; base += S.nblocks * blockDim.x) {
            const int w = base + threadIdx.x;
            double red = 0.0;
            const int plane = w / S.g.h, i = w - plane * S.g.h;
            auto at = [&](const HV &f) { return f.d + (size_t)plane * f.stride + i; };
            if (w < items) {
            // fields written earlier in this launch are read through L2 (__ldcg):
            // another SM's L1 may hold an older copy
            if (op == V_TWIST_BO) {  // t = A^-1 b_o (odd)
                const double2 b = __ldg(at(S.bo));
                const int chi = plane / 6;
                const cx<double> c = mk(S.tw_inv[chi][0], S.tw_inv[chi][1]), v = cmul(c, mk(b.x, b.y));
                *at(S.t) = make_double2(v.re, v.im);
            } else if (op == V_SETUP) {  // r = p = rhs, x_e = 0
                const double2 b = __ldcg(at(S.rhs));
                *at(S.r) = b;
                *at(S.p) = b;
                *at(S.xe) = make_double2(0.0, 0.0);
            } else if (op == V_XR) {  // x += alpha p, r -= alpha q, |r|^2
                const double a = __ldcg(&q.alpha);
                const double2 pp = __ldcg(at(S.p)), qq = __ldcg(at(S.q));
                double2 xx = __ldcg(at(S.xe)), rr = __ldcg(at(S.r));
                xx.x = fma(a, pp.x, xx.x);
                xx.y = fma(a, pp.y, xx.y);
                rr.x = fma(-a, qq.x, rr.x);
                rr.y = fma(-a, qq.y, rr.y);
                *at(S.xe) = xx;
                *at(S.r) = rr;
                red += rr.x * rr.x + rr.y * rr.y;
            } else if (op == V_P) {  // p = r + beta p
                const double bt = __ldcg(&q.beta);
                const double2 rr = __ldcg(at(S.r));
                double2 pp = __ldcg(at(S.p));
                pp.x = fma(bt, pp.x, rr.x);
                pp.y = fma(bt, pp.y, rr.y);
                *at(S.p) = pp;
            } else if (op == V_TRUE) {  // r = rhs - q (the FP64 true residual), |r|^2
                const double2 b = __ldcg(at(S.rhs)), qq = __ldcg(at(S.q));
                const double2 rr = make_double2(b.x - qq.x, b.y - qq.y);
                *at(S.r) = rr;
                red += rr.x * rr.x + rr.y * rr.y;
            } else {  // V_RESTART: p = r
                *at(S.p) = __ldcg(at(S.r));
            }
            }
            if (red_slot >= 0) {
                const double t = block_total(red);
                if (threadIdx.x == 0) x.part[(size_t)red_slot * x.nchunk + S.chunk0 + base / blockDim.x] = t;
            }
        }
    }
}

// ---- the persistent kernel

__global__ void __launch_bounds__(kManyThreads) many_cg_kernel(const ManySys *sys, ManyState *st, double *part,
                                                              const int *block_sys, int n, int nchunk, long long budget)
{
    const Ctx x{sys, st, part, block_sys, n, (int)gridDim.x, nchunk, budget};
    const int k = block_sys[blockIdx.x];
    const int lb = blockIdx.x - sys[k].block0;
    int where = 0;
#define QCD_SYNC(FIN)                                      \
    if (!grid_barrier(x, where++, [&]() { FIN; })) return;
    // ---- source: t = A^-1 b_o ; b' = b_e + kappa D_eo t ; t = A^-dag D_oe^dag b' ;
    //      rhs = A^dag b' - kappa^2 D_eo^dag t (|rhs|^2) ; r = p = rhs, x_e = 0
    vec_phase(x, k, lb, V_TWIST_BO, -1);
    QCD_SYNC(;)
    hop_phase(x, k, lb, MC_SRC_B, 0, false, &ManySys::t, &ManySys::be, &ManySys::bp, -1, false);
    QCD_SYNC(;)
    hop_phase(x, k, lb, MC_SRC_T, 1, true, &ManySys::bp, nullptr, &ManySys::t, -1, false);
    QCD_SYNC(;)
    hop_phase(x, k, lb, MC_SRC_R, 0, true, &ManySys::t, &ManySys::bp, &ManySys::rhs, 0, false);
    QCD_SYNC({
        for (int j = 0; j < x.n; ++j) {
            const double b2 = chunk_sum(x, 0, j, 8);
            if (threadIdx.x == 0) {
                ManySysState &q = x.st->s[j];
                q.b2 = q.rr = q.rr_true = b2;
                q.rr_stop = x.sys[j].tol2 * b2;
                q.alpha = q.beta = q.pAp = 0.0;
                q.iter_done = 0;
                q.status = b2 == 0.0 ? MS_DONE : (isfinite(b2) ? MS_RUNNING : MS_BREAKDOWN);
            }
        }
        if (threadIdx.x == 0) {
            x.st->iter = 0;
            x.st->reliable = 0;
        }
    })
    vec_phase(x, k, lb, V_SETUP, -1);
    QCD_SYNC(;)
    for (;;) {
        // the loop decision is read by every block after the same barrier
        bool any_run = false, any_conv = false;
        for (int j = 0; j < n; ++j) {
            const int sj = __ldcg(&st->s[j].status);
            any_run = any_run || sj == MS_RUNNING;
            any_conv = any_conv || sj == MS_CONVERGED;
        }
        if (any_run && __ldcg(&st->iter) < st->maxiter) {
            // ---- one CG iteration on the running systems
            hop_phase(x, k, lb, MC_OP1, 1, false, &ManySys::p, nullptr, &ManySys::t, -1, true);
            QCD_SYNC(;)
            hop_phase(x, k, lb, MC_OP2, 0, false, &ManySys::t, &ManySys::p, &ManySys::s, 0, true);
            QCD_SYNC({
                for (int j = 0; j < x.n; ++j) {
                    const double pAp = chunk_sum(x, 0, j, 8);
                    ManySysState &q = x.st->s[j];
                    if (threadIdx.x != 0 || q.status != MS_RUNNING) continue;
                    q.pAp = pAp;
                    if (!(pAp > 0.0) || !isfinite(pAp)) {
                        q.status = MS_BREAKDOWN;
                        q.alpha = 0.0;
                    } else {
                        q.alpha = q.rr / pAp;
                    }
                }
            })
            hop_phase(x, k, lb, MC_OP3, 1, true, &ManySys::s, nullptr, &ManySys::t, -1, true);
            QCD_SYNC(;)
            hop_phase(x, k, lb, MC_OP4, 0, true, &ManySys::t, &ManySys::s, &ManySys::q, -1, true);
            QCD_SYNC(;)
            vec_phase(x, k, lb, V_XR, 0);
            QCD_SYNC({
                if (threadIdx.x == 0) x.st->iter += 1;
                for (int j = 0; j < x.n; ++j) {
                    const double rn = chunk_sum(x, 0, j, 12);
                    ManySysState &q = x.st->s[j];
                    if (threadIdx.x != 0 || q.status != MS_RUNNING) continue;
                    if (!isfinite(rn)) {
                        q.status = MS_BREAKDOWN;
                        continue;
                    }
                    q.beta = rn / q.rr;
                    q.rr = rn;
                    if (rn <= q.rr_stop) {
                        q.status = MS_CONVERGED;
                        q.iter_done = x.st->iter;
                    }
                }
            })
            vec_phase(x, k, lb, V_P, -1);
            QCD_SYNC(;)
        } else if (any_conv) {
            // ---- FP64 true residual of the converged systems: q = Mhat^dag Mhat x_e
            //      (into q via s, t), r = rhs - q; DONE if it meets the target,
            //      else CG restarts from it
            hop_phase(x, k, lb, MC_OP1, 1, false, &ManySys::xe, nullptr, &ManySys::t, -1, false);
            QCD_SYNC(;)
            hop_phase(x, k, lb, MC_OP2, 0, false, &ManySys::t, &ManySys::xe, &ManySys::s, -1, false);
            QCD_SYNC(;)
            hop_phase(x, k, lb, MC_OP3, 1, true, &ManySys::s, nullptr, &ManySys::t, -1, false);
            QCD_SYNC(;)
            hop_phase(x, k, lb, MC_OP4, 0, true, &ManySys::t, &ManySys::s, &ManySys::q, -1, false);
            QCD_SYNC(;)
            vec_phase(x, k, lb, V_TRUE, 0);
            QCD_SYNC({
                if (threadIdx.x == 0) x.st->reliable += 1;
                for (int j = 0; j < x.n; ++j) {
                    const double rt = chunk_sum(x, 0, j, 12);
                    ManySysState &q = x.st->s[j];
                    if (threadIdx.x != 0 || q.status != MS_CONVERGED) continue;
                    q.rr_true = rt;
                    if (!isfinite(rt)) {
                        q.status = MS_BREAKDOWN;
                    } else if (rt <= q.rr_stop) {
                        q.status = MS_DONE;
                    } else {
                        // restart from the true residual (still CONVERGED for the next phase)
                        q.rr = rt;
                        q.beta = 0.0;
                    }
                }
            })
            vec_phase(x, k, lb, V_RESTART, -1);
            QCD_SYNC({
                if (threadIdx.x == 0)
                    for (int j = 0; j < x.n; ++j)
                        if (x.st->s[j].status == MS_CONVERGED) x.st->s[j].status = MS_RUNNING;
            })
        } else {
            break;
        }
    }
    // ---- odd sites x_o = A^-1 b_o + kappa A^-1 D_oe x_e, then |b - M x|^2, |b|^2
    hop_phase(x, k, lb, MC_RECON, 1, false, &ManySys::xe, &ManySys::bo, &ManySys::xo, -1, false);
    QCD_SYNC(;)
    // M x per parity: out = A x - kappa D x (even from x_o, odd from x_e)
    hop_phase(x, k, lb, MC_FULL, 0, false, &ManySys::xo, &ManySys::xe, nullptr, 0, false);
    hop_phase(x, k, lb, MC_FULL, 1, false, &ManySys::xe, &ManySys::xo, nullptr, 1, false);
    bnorm_phase(x, k, lb, 2);
    QCD_SYNC({
        for (int j = 0; j < x.n; ++j) {
            const double r0 = chunk_sum(x, 0, j, 8);
            const double r1 = chunk_sum(x, 1, j, 8);
            const double b2 = chunk_sum(x, 2, j, 24);
            if (threadIdx.x != 0) continue;
            ManySysState &q = x.st->s[j];
            q.full_r2 = r0 + r1;
            q.full_b2 = b2;
            if (q.status == MS_RUNNING || q.status == MS_CONVERGED) q.status = MS_MAXITER;
        }
    })
#undef QCD_SYNC
}

void put(PhaseCoef &pc, const Coef &cy, const Coef &cd)
{
    memcpy(pc.cy, cy.c, sizeof(pc.cy));
    memcpy(pc.cd, cd.c, sizeof(pc.cd));
}

}  // namespace
}  // namespace qcd

using namespace qcd;

extern "C" qcd_status qcd_solve_cg_many(int n, const qcd_gauge *const *gauges, qcd_spinor *const *x,
                                        const qcd_spinor *const *b, const qcd_solver_params *prm,
                                        qcd_solver_stats *stats, long long wait_cycles, int max_blocks,
                                        void *stream)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (n < 1 || n > kManyMax) return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: n = %d not in 1..%d", n, kManyMax);
    if (!gauges || !x || !b || !prm) return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: NULL argument");
    for (int k = 0; k < n; ++k) {
        const qcd_gauge *g = gauges[k];
        if (!g || !x[k] || !b[k]) return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: NULL handle (system %d)", k);
        if (g->prec != QCD_PREC_F64) return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: gauge field %d must be F64", k);
        // x and b live on the gauge field's lattice or on a context lattice of
        // the same extents (whose handle then holds this system's scratch)
        const qcd_lattice *xl = x[k]->lat;
        if (b[k]->lat != xl || memcmp(xl->dims, g->lat->dims, sizeof(xl->dims)) != 0 || xl->t_bc != g->lat->t_bc)
            return fail(QCD_ERR_INVALID_ARG,
                        "solve_cg_many: x and b of system %d must share a lattice with the gauge field's extents", k);
        if (x[k]->parity != QCD_PARITY_FULL || b[k]->parity != QCD_PARITY_FULL || x[k]->prec != QCD_PREC_F64 ||
            b[k]->prec != QCD_PREC_F64 || x[k]->ks || b[k]->ks)
            return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: x and b must be FULL F64 Wilson fields (system %d)", k);
        if (x[k]->data == b[k]->data) return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: x aliases b (system %d)", k);
        for (int j = 0; j < k; ++j)
            if (x[j]->data == x[k]->data) return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: systems %d and %d share x", j, k);
        const qcd_solver_params &q = prm[k];
        if (!q.eo || q.normal || q.inner_prec != QCD_PREC_F64)
            return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: even-odd FP64 CG only (eo = 1, normal = 0, inner F64; system %d)", k);
        if (!(q.tol > 0.0) || q.maxiter < 1 || q.maxiter > (1 << 30) || !std::isfinite(q.kappa) || !std::isfinite(q.mu))
            return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: bad tol/maxiter/kappa/mu (system %d)", k);
        if (q.maxiter != prm[0].maxiter)
            return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: the systems share one maxiter (system %d)", k);
    }
    if (wait_cycles < 0) return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: wait_cycles must be >= 0");
    if (max_blocks < 0 || (max_blocks > 0 && max_blocks < n))
        return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: max_blocks = %d must be 0 or at least n = %d", max_blocks, n);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0, per_sm = 0, coop = 0;
    QCD_CHECK_CUDA(cudaGetDevice(&dev), "solve_cg_many");
    QCD_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "solve_cg_many");
    QCD_CHECK_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev), "solve_cg_many");
    if (!coop) return fail(QCD_ERR_CUDA, "solve_cg_many: the device has no cooperative launch");
    QCD_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, many_cg_kernel, kManyThreads, 0),
                   "solve_cg_many: occupancy");
    if (per_sm < 1) return fail(QCD_ERR_CUDA, "solve_cg_many: the kernel does not fit an SM");
    // blocks: every block resident (cooperative launch), divided among the
    // systems in proportion to their sites, at least one each, and no more
    // than a system can use (8 threads per site)
    long long total_h = 0;
    for (int k = 0; k < n; ++k) total_h += x[k]->lat->h;
    // every block resident at once; a caller sharing the GPU with other work
    // may ask for fewer (max_blocks), so the launch need not wait for the
    // whole GPU to drain
    const int grid_cap = max_blocks > 0 ? std::min(max_blocks, nsm * per_sm) : nsm * per_sm;
    std::vector<int> nb(n);
    int used = 0;
    for (int k = 0; k < n; ++k) {
        const int h = x[k]->lat->h;
        const int useful = std::max(1, (8 * h + kManyThreads - 1) / kManyThreads);
        nb[k] = std::max(1, std::min(useful, (int)((long long)(grid_cap - n) * h / total_h)));
        used += nb[k];
    }
    if (used > grid_cap) return fail(QCD_ERR_INVALID_ARG, "solve_cg_many: too many systems for one resident grid");
    std::vector<ManySys> hs(n);
    std::vector<int> block_sys;
    int nchunk = 0;  // reduction chunks per partial slot, all systems
    const qcd_lattice *lat0 = x[0]->lat;
    for (int k = 0; k < n; ++k) {
        const qcd_gauge *g = gauges[k];
        const qcd_lattice *lat = x[k]->lat;
        qcd_status st = QCD_OK;
        const GaugeView U = gauge_view(g, QCD_PREC_F64, 18, s, &st);
        if (st != QCD_OK) return st;
        ManySys &S = hs[k];
        memset(&S, 0, sizeof(S));
        S.g = lat->geom;
        S.U = static_cast<const double2 *>(U.data);
        S.ustride = U.stride;
        auto half = [&](const qcd_spinor *f, int h) {
            return HV{reinterpret_cast<double2 *>(static_cast<char *>(f->data) + h * f->half_data_bytes), lat->stride};
        };
        S.be = half(b[k], 0);
        S.bo = half(b[k], 1);
        S.xe = half(x[k], 0);
        S.xo = half(x[k], 1);
        const char *names[7] = {"bp", "rhs", "r", "p", "q", "t", "s"};
        HV *dst[7] = {&S.bp, &S.rhs, &S.r, &S.p, &S.q, &S.t, &S.s};
        for (int f = 0; f < 7; ++f) {
            const FieldView v = ws_field(lat, std::string("many") + std::to_string(k) + "_" + names[f], 1, QCD_PREC_F64);
            if (!v.hv[0].data) return fail(QCD_ERR_OOM, "solve_cg_many: workspace");
            *dst[f] = HV{static_cast<double2 *>(v.hv[0].data), v.hv[0].stride};
        }
        const double kappa = prm[k].kappa, a = 2.0 * kappa * prm[k].mu;
        const Coef zero = coef_real(0.0);
        memcpy(S.tw_inv, coef_twist_inv(a).c, sizeof(S.tw_inv));
        put(S.pc[MC_SRC_B], coef_real(1.0), coef_real(kappa));
        put(S.pc[MC_SRC_T], zero, coef_twist_inv(-a));
        put(S.pc[MC_SRC_R], coef_twist(-a), coef_real(-kappa * kappa));
        put(S.pc[MC_OP1], zero, coef_twist_inv(a));
        put(S.pc[MC_OP2], coef_twist(a), coef_real(-kappa * kappa));
        put(S.pc[MC_OP3], zero, coef_twist_inv(-a));
        put(S.pc[MC_OP4], coef_twist(-a), coef_real(-kappa * kappa));
        put(S.pc[MC_RECON], coef_twist_inv(a), coef_scale(coef_twist_inv(a), kappa));
        put(S.pc[MC_FULL], coef_twist(a), coef_real(-kappa));
        S.tol2 = prm[k].tol * prm[k].tol;
        S.block0 = (int)block_sys.size();
        S.chunk0 = nchunk;
        nchunk += (24 * lat->h + kManyThreads - 1) / kManyThreads;
        S.nblocks = nb[k];
        for (int j = 0; j < nb[k]; ++j) block_sys.push_back(k);
    }
    const int grid = (int)block_sys.size();
    // device-side descriptors, state and partials (workspace of the first
    // system's lattice; the host copies are staged in pageable memory and
    // the stream is synchronised before this call returns)
    const size_t desc_bytes = sizeof(ManySys) * n, bs_bytes = sizeof(int) * grid, st_bytes = sizeof(ManyState),
                 part_bytes = sizeof(double) * 3 * (size_t)nchunk;
    char *ws = static_cast<char *>(workspace(lat0, "many_ctl", desc_bytes + bs_bytes + st_bytes + part_bytes + 1024));
    if (!ws) return fail(QCD_ERR_OOM, "solve_cg_many: workspace");
    auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
    ManySys *d_sys = reinterpret_cast<ManySys *>(ws);
    int *d_bs = reinterpret_cast<int *>(ws + align(desc_bytes));
    ManyState *d_st = reinterpret_cast<ManyState *>(ws + align(desc_bytes) + align(bs_bytes));
    double *d_part = reinterpret_cast<double *>(ws + align(desc_bytes) + align(bs_bytes) + align(st_bytes));
    ManyState h_st;
    memset(&h_st, 0, sizeof(h_st));
    h_st.n = n;
    h_st.maxiter = prm[0].maxiter;
    QCD_CHECK_CUDA(cudaMemcpyAsync(d_sys, hs.data(), desc_bytes, cudaMemcpyHostToDevice, s), "solve_cg_many");
    QCD_CHECK_CUDA(cudaMemcpyAsync(d_bs, block_sys.data(), bs_bytes, cudaMemcpyHostToDevice, s), "solve_cg_many");
    QCD_CHECK_CUDA(cudaMemcpyAsync(d_st, &h_st, sizeof(h_st), cudaMemcpyHostToDevice, s), "solve_cg_many");
    long long budget = wait_cycles > 0 ? wait_cycles : 4000000000LL;  // ~2 s at 2 GHz
    int nn = n, nc = nchunk;
    void *args[] = {&d_sys, &d_st, &d_part, &d_bs, &nn, &nc, &budget};
    QCD_CHECK_CUDA(cudaLaunchCooperativeKernel((const void *)many_cg_kernel, dim3(grid), dim3(kManyThreads), args, 0, s),
                   "solve_cg_many: launch");
    note_launches();
    QCD_CHECK_CUDA(cudaMemcpyAsync(&h_st, d_st, sizeof(h_st), cudaMemcpyDeviceToHost, s), "solve_cg_many");
    QCD_CHECK_CUDA(cudaStreamSynchronize(s), "solve_cg_many");
    if (h_st.error == QCD_ERR_TIMEOUT)
        return fail(QCD_ERR_TIMEOUT, "solve_cg_many: a grid barrier wait ran out of its %lld-cycle budget (phase %d)",
                    budget, h_st.timeout_where);
    qcd_status result = QCD_OK;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < n; ++k) {
        const ManySysState &q = h_st.s[k];
        if (q.status == MS_BREAKDOWN)
            result = fail(QCD_ERR_BREAKDOWN, "solve_cg_many: breakdown in system %d", k);
        else if (q.status != MS_DONE && result == QCD_OK)
            result = fail(QCD_ERR_NOT_CONVERGED, "solve_cg_many: maxiter reached (system %d)", k);
        if (stats) {
            stats[k].iterations = q.status == MS_DONE ? q.iter_done : h_st.iter;
            stats[k].reliable_updates = h_st.reliable;
            stats[k].true_rel_residual = q.b2 > 0.0 ? std::sqrt(q.rr_true / q.b2) : 0.0;
            stats[k].full_rel_residual = q.full_b2 > 0.0 ? std::sqrt(q.full_r2 / q.full_b2) : 0.0;
            stats[k].seconds = secs;
        }
    }
    return result;
}
