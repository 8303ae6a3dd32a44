// Conjugate-gradient inversion of the Wilson / twisted-mass Wilson matrix.
//
// CL2QCD (arXiv:1411.5219, Sec. 1) inverts the fermion matrix D phi = psi
// with Krylov methods such as CG, applying D many times.  Here:
//
//   even-odd (eo = 1):  b'_e = b_e + kappa D_eo A^-1 b_o
//                       CG on Mhat^dag Mhat x_e = Mhat^dag b'_e
//                       x_o  = A^-1 (b_o + kappa D_oe x_e)
//   full (eo = 0):      CG on M^dag M x = b (normal) or M^dag b
//
// CG is Hestenes-Stiefel with alpha = |r|^2 / |Mhat p|^2 (the CGNR form of
// <p, Mhat^dag Mhat p>), fused into the operator's last-but-one kernel.
// Scalars live on the device (CgState): the host enqueues batches of
// iterations and reads the state back once per batch.  A converged or
// reliable-update state stops the batch; the host then recomputes the
// residual in FP64 from the accumulated solution (true residual), which
// either confirms convergence or replaces the iterated residual and
// continues.  In mixed precision the inner iterations run on
// FP32/FP16/BF16 fields and links (FP32 arithmetic), the solution
// correction accumulates in FP32 and is added to the FP64 solution at each
// reliable update (Sleijpen and van der Vorst's reliable-update scheme).
#include <chrono>
#include <cmath>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "qcd_handles.h"

namespace qcd {
namespace {

struct OpCtx {
    const qcd_lattice *lat;
    bool tw;               // some right-hand side has mu != 0 (complex chiral coefficients)
    bool eo;
    const Reduction *red;  // scratch of the fused |Mhat p|^2 reduction
    const double *coef;    // device table of the epilogue coefficients, kCoefPerRhs doubles per rhs
    const float *coef_f;   // the same table rounded to float (read by the FP32 and 16-bit kernels)
};

// Per right-hand side, the solve reads every kappa- and mu-dependent
// coefficient from one device table, so a batch may mix kappa and mu values
// and the cached CG graph depends on neither.  Blocks of 8 doubles
// (cy[2][2], cd[2][2]) at these offsets:
constexpr int kCoefPerRhs = 96;
constexpr int kMaxIter = 1 << 30;  // largest accepted maxiter
constexpr int kCoefOp = 0;        // normal operator, 4 hops (2 for the full lattice)
constexpr int kCoefSrcB = 32;     // b' = b_e + kappa D_eo A^-1 b_o
constexpr int kCoefSrcT = 40;     // t = A^-dag D_oe^dag b'
constexpr int kCoefSrcR = 48;     // rhs = A^dag b' - kappa^2 D_eo^dag t
constexpr int kCoefRecon = 56;    // x_o = A^-1 b_o + kappa A^-1 D_oe x_e
constexpr int kCoefFullM = 64;    // M = A - kappa D
constexpr int kCoefFullMd = 72;   // M^dag
constexpr int kCoefTwistInv = 80; // A^-1 (4 doubles: one complex per chirality)

void put_coef(double *t, int off, const Coef &cy, const Coef &cd)
{
    memcpy(t + off, cy.c, 4 * sizeof(double));
    memcpy(t + off + 4, cd.c, 4 * sizeof(double));
}

// The coefficient block of one right-hand side with hopping parameter
// kappa and a = 2 kappa mu.
void coef_block(double *t, bool eo, double kappa, double a)
{
    const Coef zero = coef_real(0.0);
    if (eo) {
        put_coef(t, kCoefOp + 0, zero, coef_twist_inv(a));
        put_coef(t, kCoefOp + 8, coef_twist(a), coef_real(-kappa * kappa));
        put_coef(t, kCoefOp + 16, zero, coef_twist_inv(-a));
        put_coef(t, kCoefOp + 24, coef_twist(-a), coef_real(-kappa * kappa));
    } else {
        put_coef(t, kCoefOp + 0, coef_twist(a), coef_real(-kappa));
        put_coef(t, kCoefOp + 8, coef_twist(-a), coef_real(-kappa));
    }
    put_coef(t, kCoefSrcB, coef_real(1.0), coef_real(kappa));
    put_coef(t, kCoefSrcT, zero, coef_twist_inv(-a));
    put_coef(t, kCoefSrcR, coef_twist(-a), coef_real(-kappa * kappa));
    put_coef(t, kCoefRecon, coef_twist_inv(a), coef_scale(coef_twist_inv(a), kappa));
    put_coef(t, kCoefFullM, coef_twist(a), coef_real(-kappa));
    put_coef(t, kCoefFullMd, coef_twist(-a), coef_real(-kappa));
    const Coef ti = coef_twist_inv(a);
    memcpy(t + kCoefTwistInv, ti.c, 4 * sizeof(double));
}

// The reliable-update factor for reliable_delta = 0.  Between two FP64
// updates the inner iteration reduces the residual by 1/delta; its drift
// from the true residual grows with the inner format's rounding unit u, so
// delta stays well above u: about 20 u for FP16 (u = 2^-11); 1e-3 for FP32
// and 1e-4 for DF64, far above theirs; 0.1 for BF16 (u = 2^-8), which needed
// more iterations at 0.01 and stalled at 0.003.  Measured on the 24^3x8,
// 32^3x8 and 48^3x12 workloads: FP16 at 0.01 takes 5 updates instead of 9
// at 0.1 with the same iteration count (48^3x12: 33.0 ms against 42.7 ms).
double default_reliable_delta(int inner_prec)
{
    switch (inner_prec) {
    case QCD_PREC_F32: return 1e-3;
    case QCD_PREC_F16: return 1e-2;
    case QCD_PREC_DF64: return 1e-4;
    default: return 0.1;
    }
}

// A hop whose epilogue coefficients come from block `off` of the table.
HopArgs table_hop(const OpCtx &c, int off)
{
    HopArgs h{};
    h.coef = c.coef + off;
    h.coef_f = c.coef_f + off;
    h.coef_stride = kCoefPerRhs;
    h.twisted = c.tw;
    return h;
}

// How the kernels of one operator application run.
struct OpRun {
    bool check = false;              // early exit unless the CG state is run_status
    int run_status = CG_RUNNING;
    bool reduce = false;             // |out|^2 of the last kernel -> fin
    FinalizeKind fin = FIN_STORE;
};

HopArgs op_hop(const OpCtx &c, int off, const OpRun &r)
{
    HopArgs h = table_hop(c, off);
    h.check_status = r.check;
    h.run_status = r.run_status;
    h.fin = r.fin;
    return h;
}

// out = Mhat in (eo; t: odd-site temporary) or M in (full).
cudaError_t apply_fwd(const OpCtx &c, const GaugeView &U, int recon, const FieldView &in, const FieldView &out,
                      const FieldView &t, const OpRun &r, cudaStream_t st)
{
    cudaError_t e;
    if (c.eo) {
        HopArgs h = op_hop(c, kCoefOp + 0, r);  // t = A^-1 D_oe in
        h.out = &t;
        h.in = &in;
        h.out_parity = 1;
        h.plain = !c.tw;
        if ((e = hop(c.lat, U, recon, h, st)) != cudaSuccess) return e;
        HopArgs h2 = op_hop(c, kCoefOp + 8, r);  // out = A in - kappa^2 D_eo t
        h2.out = &out;
        h2.in = &t;
        h2.y = &in;
        h2.out_parity = 0;
        h2.reduce = r.reduce;
        h2.red = c.red;
        return hop(c.lat, U, recon, h2, st);
    }
    HopArgs h = op_hop(c, kCoefOp + 0, r);  // out = A in - kappa D in
    h.out = &out;
    h.in = &in;
    h.y = &in;
    h.both = true;
    h.reduce = r.reduce;
    h.red = c.red;
    return hop(c.lat, U, recon, h, st);
}

// out = Mhat^dag in (eo; t: odd-site temporary) or M^dag in (full).
cudaError_t apply_dag(const OpCtx &c, const GaugeView &U, int recon, const FieldView &in, const FieldView &out,
                      const FieldView &t, const OpRun &r, cudaStream_t st)
{
    cudaError_t e;
    if (c.eo) {
        HopArgs h = op_hop(c, kCoefOp + 16, r);  // t = A^-dag D_oe^dag in
        h.out = &t;
        h.in = &in;
        h.out_parity = 1;
        h.dagger = 1;
        h.plain = !c.tw;
        if ((e = hop(c.lat, U, recon, h, st)) != cudaSuccess) return e;
        HopArgs h2 = op_hop(c, kCoefOp + 24, r);  // out = A^dag in - kappa^2 D_eo^dag t
        h2.out = &out;
        h2.in = &t;
        h2.y = &in;
        h2.out_parity = 0;
        h2.dagger = 1;
        h2.reduce = r.reduce;
        h2.red = c.red;
        return hop(c.lat, U, recon, h2, st);
    }
    HopArgs h = op_hop(c, kCoefOp + 8, r);  // out = M^dag in
    h.out = &out;
    h.in = &in;
    h.y = &in;
    h.both = true;
    h.dagger = 1;
    h.reduce = r.reduce;
    h.red = c.red;
    return hop(c.lat, U, recon, h, st);
}

// out = Mhat^dag Mhat in (eo) or M^dag M in (full).  t (odd half) and s
// (even half, or full) are temporaries of the same precision.  With
// reduce_alpha the second kernel also reduces |Mhat in|^2 into alpha.
cudaError_t apply_normal(const OpCtx &c, const GaugeView &U, int recon, const FieldView &in, const FieldView &out,
                         const FieldView &t, const FieldView &s, bool reduce_alpha, bool check, cudaStream_t st)
{
    OpRun r;
    r.check = check;
    r.reduce = reduce_alpha;
    r.fin = FIN_CG_ALPHA;
    cudaError_t e = apply_fwd(c, U, recon, in, s, t, r, st);
    if (e != cudaSuccess) return e;
    r.reduce = false;
    return apply_dag(c, U, recon, s, out, t, r, st);
}

// out = M in on a full field (dagger: M^dag).
cudaError_t apply_full_m(const OpCtx &c, const GaugeView &U, int recon, const FieldView &in, const FieldView &out,
                         int dagger, cudaStream_t st)
{
    HopArgs h = table_hop(c, dagger ? kCoefFullMd : kCoefFullM);
    h.fin = FIN_STORE;
    h.out = &out;
    h.in = &in;
    h.y = &in;
    h.both = true;
    h.dagger = dagger;
    return hop(c.lat, U, recon, h, st);
}


// Everything one CG loop needs: operator context, gauge views, the FP64 and
// inner fields, the reduction scratch and the device state.
struct CgFields {
    OpCtx c;
    GaugeView Uh, Us;
    int rh_recon, rs_recon;
    bool mixed;
    FieldView rhs, xh, rh, qh, th, sh;  // FP64
    FieldView rs, ps, qs, ts, ss, xs;   // inner (aliases of the FP64 ones when not mixed)
    Reduction red;
    CgState *state;
    // Split true residual (mixed precision with an un-normalised system
    // rhs0: b'_e for eo, b for the full-lattice M^dag M x = M^dag b): the
    // FP64 defect rho = rhs0 - Mhat x is mapped by Mhat^dag in a lower
    // precision; only an estimate that meets the target is checked with the
    // FP64 Mhat^dag.
    bool split;
    FieldView rhs0;
    // The precision of the defect's Mhat^dag image: FP32 for 16-bit inner
    // fields (a 16-bit image would carry cond(Mhat) times the 16-bit
    // roundoff), else the inner precision.  With FP32 it is cast to the inner
    // r once.
    GaugeView Um;
    int rm_recon;
    bool mid;               // the image has its own FP32 fields
    FieldView rho_m, t_m, r_m;
};

// One CG iteration: q = A p (|Mhat p|^2 -> alpha), x += alpha p, r -= alpha q
// (|r|^2 -> beta and status), p = r + beta p.  All return at once unless
// the state is RUNNING.
cudaError_t enqueue_iteration(const CgFields &f, cudaStream_t s)
{
    cudaError_t e = apply_normal(f.c, f.Us, f.rs_recon, f.ps, f.qs, f.ts, f.ss, true, true, s);
    if (e == cudaSuccess) e = launch_cg_xr(f.mixed ? f.xs : f.xh, f.ps, f.rs, f.qs, f.red, f.state, s);
    if (e == cudaSuccess) e = launch_cg_p(f.ps, f.rs, f.state, s);
    return e;
}

// Reliable update / convergence check: x += xs (mixed), r = rhs - A x in
// FP64 (|r|^2 -> DONE or RUNNING with beta = |r|^2 / |r_prev|^2), r_inner =
// cast(r), then p = r + beta p.
cudaError_t enqueue_true_residual(const CgFields &f, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (f.split) {
        // x += xs; rho = rhs0 - Mhat x (FP64, two hops); r_inner = Mhat^dag rho
        // in FP32 or the inner precision (two hops, |r|^2 -> estimate); under
        // CG_VERIFY the FP64 Mhat^dag rho and its norm decide; then p = r + beta p.
        OpRun plain_run;
        OpRun est;
        est.reduce = true;
        est.fin = FIN_CG_TRUE_EST;
        OpRun check;
        check.check = true;
        check.run_status = CG_VERIFY;
        e = launch_cg_accum_x(f.xh, f.xs, s);
        if (e == cudaSuccess) e = apply_fwd(f.c, f.Uh, f.rh_recon, f.xh, f.sh, f.th, plain_run, s);
        if (f.mid) {
            if (e == cudaSuccess) e = launch_cg_defect(f.rhs0, f.sh, f.rh, f.rho_m, s);
            if (e == cudaSuccess) e = apply_dag(f.c, f.Um, f.rm_recon, f.rho_m, f.r_m, f.t_m, est, s);
            if (e == cudaSuccess) e = launch_convert(f.rs, f.r_m, s);
        } else {
            if (e == cudaSuccess) e = launch_cg_defect(f.rhs0, f.sh, f.rh, f.ss, s);
            if (e == cudaSuccess) e = apply_dag(f.c, f.Us, f.rs_recon, f.ss, f.rs, f.ts, est, s);
        }
        if (e == cudaSuccess) e = apply_dag(f.c, f.Uh, f.rh_recon, f.rh, f.qh, f.th, check, s);
        if (e == cudaSuccess) e = launch_cg_verify(f.qh, f.red, f.state, s);
        if (e == cudaSuccess) e = launch_cg_p(f.ps, f.rs, f.state, s);
        return e;
    }
    if (f.mixed) e = launch_cg_accum_x(f.xh, f.xs, s);
    if (e == cudaSuccess) e = apply_normal(f.c, f.Uh, f.rh_recon, f.xh, f.qh, f.th, f.sh, false, false, s);
    if (e == cudaSuccess) e = launch_cg_true_residual(f.rhs, f.qh, f.rh, f.mixed ? &f.rs : nullptr, f.red, f.state, s);
    if (e == cudaSuccess) e = launch_cg_p(f.ps, f.rs, f.state, s);
    return e;
}

cudaError_t read_state(const qcd_lattice *lat, cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(lat->state_host, lat->state, sizeof(CgState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

// Host-driven loop: batches of iterations, the state read back after each.
// The batch is sized from the observed convergence rate to end near the
// next reliable update (mixed) or the target residual.
cudaError_t cg_eager(const qcd_lattice *lat, const CgFields &f, cudaStream_t s)
{
    // the slowest running right-hand side sets the pace: its log distance to
    // the target (and to the next reliable update) in residual^2
    auto distance = [](const CgState &st) {
        double d = 0.0;
        for (int k = 0; k < st.nrhs; ++k) {
            const CgRhs &q = st.r[k];
            if (q.status != CG_RUNNING || q.rr <= 0.0) continue;
            double dk = std::log(q.rr / q.rr_stop);
            if (st.delta2 > 0.0) dk = std::min(dk, std::log(q.rr / (st.delta2 * q.rr_max)));
            d = std::max(d, dk);
        }
        return d;
    };
    cudaError_t e = read_state(lat, s);
    if (e != cudaSuccess) return e;
    int batch = 2;
    double last_d = distance(*lat->state_host);
    int last_iter = 0;
    for (;;) {
        const int status = lat->state_host->status;
        if (status == CG_DONE || status == CG_BREAKDOWN || status == CG_MAXITER) return cudaSuccess;
        if (status == CG_CONVERGED || status == CG_RELIABLE)
            if ((e = enqueue_true_residual(f, s)) != cudaSuccess) return e;
        for (int k = 0; k < batch; ++k)
            if ((e = enqueue_iteration(f, s)) != cudaSuccess) return e;
        if ((e = read_state(lat, s)) != cudaSuccess) return e;
        const CgState &hs = *lat->state_host;
        const int done = hs.iter - last_iter;
        const double d = distance(hs);
        if (done > 0 && hs.status == CG_RUNNING && last_d > d && d > 0.0) {
            const double rate = (last_d - d) / done;
            batch = (int)std::min(64.0, std::max(1.0, std::ceil(d / rate)));
        } else {
            batch = std::max(1, std::min(8, batch));
        }
        last_d = d;
        last_iter = hs.iter;
    }
}

// The CG loop as one CUDA graph: a WHILE node whose body runs one iteration,
// then an IF node that runs the reliable update when the iteration asked
// for it, then a control kernel that keeps the loop going while the state
// is RUNNING (bounded by iter < maxiter and a trip cap).  Built once per
// configuration and field addresses and cached on the lattice.
qcd_status cg_graph(const qcd_lattice *lat, const CgFields &f, cudaGraphExec_t *out)
{
    char key[512];
    snprintf(key, sizeof(key), "%d|%d|%p|%d|%d|%d|%p|%p|%p|%p|%p|%p|%p|%p|%p|%p|%p|%p|%p|%p|%d|%d", (int)f.c.eo,
             (int)f.c.tw, (const void *)f.c.coef, (int)f.mixed, f.rh_recon, f.rs_recon, f.Uh.data, f.Us.data, f.rhs.hv[0].data,
             f.xh.hv[0].data, f.xh.hv[1].data, f.rh.hv[0].data, f.qh.hv[0].data, f.th.hv[0].data, f.sh.hv[0].data,
             f.rs.hv[0].data, f.ps.hv[0].data, f.qs.hv[0].data, f.ts.hv[0].data, f.ss.hv[0].data, f.xs.hv[0].data,
             (void *)f.state, f.rs.prec, f.rhs.nh);
    const size_t used = strlen(key);
    snprintf(key + used, sizeof(key) - used, "|%p|%d|%d|%p|%d|%p|%p", (void *)f.red.partials, f.rs.rhs_log2,
             (int)f.split, f.rhs0.hv[0].data, (int)f.mid, f.Um.data, f.r_m.hv[0].data);
    auto it = lat->graphs.find(key);
    if (it != lat->graphs.end()) {
        it->second.last_use = ++lat->graph_clock;
        *out = it->second.exec;
        return QCD_OK;
    }
    if (!lat->capture_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&lat->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return check_cuda(e, "solve_cg: capture stream");
    }
    cudaStream_t cs = lat->capture_stream;
    CaptureLock cl(device_mutex());  // no device-wide call may run during the capture
    cudaGraph_t g = nullptr, tmp = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle hloop, hrel;
    cudaGraphNode_t wnode, inode;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaStreamCaptureStatus cst;
    std::vector<cudaGraphNode_t> tail;
    cudaError_t e = cudaGraphCreate(&g, 0);
#define G_TRY(x)                    \
    if (e == cudaSuccess) e = (x);
    G_TRY(cudaGraphConditionalHandleCreate(&hloop, g, 1, cudaGraphCondAssignDefault));
    G_TRY(cudaGraphConditionalHandleCreate(&hrel, g, 0, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp{};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hloop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    G_TRY(cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp));
    cudaGraph_t body = e == cudaSuccess ? wp.conditional.phGraph_out[0] : nullptr;
    // body: one iteration, then the reliable-update decision
    G_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (e == cudaSuccess) {
        cudaError_t ec = enqueue_iteration(f, cs);
        if (ec == cudaSuccess) ec = launch_cg_ctrl_reliable(f.state, hrel, cs);
        if (ec == cudaSuccess) ec = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
        if (ec == cudaSuccess && cst != cudaStreamCaptureStatusActive) ec = cudaErrorStreamCaptureInvalidated;
        if (ec == cudaSuccess && ndeps > 0 && !deps) ec = cudaErrorStreamCaptureInvalidated;
        if (ec == cudaSuccess) tail.assign(deps, deps + ndeps);
        cudaError_t ee = cudaStreamEndCapture(cs, &tmp);
        e = ec != cudaSuccess ? ec : ee;
    }
    cudaGraphNodeParams ip{};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hrel;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    G_TRY(cudaGraphAddNode(&inode, body, tail.data(), nullptr, tail.size(), &ip));
    if (e == cudaSuccess) {
        cudaGraph_t ibody = ip.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cs, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t ec = enqueue_true_residual(f, cs);
            cudaError_t ee = cudaStreamEndCapture(cs, &tmp);
            e = ec != cudaSuccess ? ec : ee;
        }
    }
    // after the IF node: the loop condition
    G_TRY(cudaStreamBeginCaptureToGraph(cs, body, &inode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    if (e == cudaSuccess) {
        cudaError_t ec = launch_cg_ctrl_loop(f.state, hloop, cs);
        cudaError_t ee = cudaStreamEndCapture(cs, &tmp);
        e = ec != cudaSuccess ? ec : ee;
    }
    G_TRY(cudaGraphInstantiate(&exec, g, 0));
#undef G_TRY
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return check_cuda(e, "solve_cg: graph build");
    }
    // keep at most 16 graphs per lattice
    if (lat->graphs.size() >= 16) {
        auto old = lat->graphs.begin();
        for (auto i = lat->graphs.begin(); i != lat->graphs.end(); ++i)
            if (i->second.last_use < old->second.last_use) old = i;
        cudaGraphExecDestroy(old->second.exec);
        cudaGraphDestroy(old->second.graph);
        lat->graphs.erase(old);
    }
    lat->graphs[key] = qcd_lattice::GraphEntry{g, exec, ++lat->graph_clock};
    *out = exec;
    return QCD_OK;
}

}  // namespace
}  // namespace qcd

using namespace qcd;

#define QCD_TRY(expr, what)                                   \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return check_cuda(e_, what);   \
    } while (0)

namespace {

FieldView half_of(const FieldView &f, int k)
{
    FieldView v = f;
    v.nh = 1;
    v.hv[0] = v.hv[1] = f.hv[k];
    return v;
}

// The solve for nrhs right-hand sides in one batched CG (nrhs = 1: the
// caller's fields are used in place).
}  // namespace

// The solve for nrhs right-hand sides in one batched CG (nrhs = 1: the
// caller's fields are used in place).  `ctx` is the lattice handle whose
// scratch, CG state and graph cache the solve uses (nullptr: the gauge
// field's own); it must have the gauge field's extents, and x, b must live
// on it.  Separate contexts let solves that share one resident gauge field
// run concurrently on different streams.
qcd_status qcd::solve_impl(const qcd_gauge *g, qcd_spinor *const *x, const qcd_spinor *const *b, int nrhs,
                      const qcd_solver_params *prm, qcd_solver_stats *stats, cudaStream_t s, const qcd_lattice *ctx)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (!g || !x || !b || !prm) return fail(QCD_ERR_INVALID_ARG, "solve_cg: NULL argument");
    if (nrhs < 1 || nrhs > kMaxRhs) return fail(QCD_ERR_INVALID_ARG, "solve_cg: nrhs = %d not in 1..%d", nrhs, kMaxRhs);
    const qcd_lattice *lat = ctx ? ctx : g->lat;
    if (memcmp(lat->dims, g->lat->dims, sizeof(lat->dims)) != 0 || lat->t_bc != g->lat->t_bc)
        return fail(QCD_ERR_INVALID_ARG, "solve_cg: the context lattice differs from the gauge field's");
    for (int k = 0; k < nrhs; ++k) {
        if (!x[k] || !b[k]) return fail(QCD_ERR_INVALID_ARG, "solve_cg: NULL field");
        if (x[k]->lat != lat || b[k]->lat != lat) return fail(QCD_ERR_INVALID_ARG, "solve_cg: lattices differ");
        if (x[k]->parity != QCD_PARITY_FULL || b[k]->parity != QCD_PARITY_FULL || x[k]->prec != QCD_PREC_F64 ||
            b[k]->prec != QCD_PREC_F64)
            return fail(QCD_ERR_INVALID_ARG, "solve_cg: x and b must be FULL F64 fields");
        if (x[k]->data == b[k]->data) return fail(QCD_ERR_INVALID_ARG, "solve_cg: x aliases b");
        if (x[k]->ks || b[k]->ks) return fail(QCD_ERR_INVALID_ARG, "solve_cg: staggered fields are not solved here");
    }
    if (g->prec != QCD_PREC_F64) return fail(QCD_ERR_INVALID_ARG, "solve_cg: the gauge field must be F64");
    for (int k = 0; k < nrhs; ++k) {
        const qcd_solver_params &q = prm[k];
        // the device loop's trip cap is maxiter + 64 in 32-bit arithmetic
        if (!(q.tol > 0.0) || q.maxiter < 1 || q.maxiter > kMaxIter || !std::isfinite(q.kappa) ||
            !std::isfinite(q.mu))
            return fail(QCD_ERR_INVALID_ARG, "solve_cg: bad tol/maxiter/kappa/mu (system %d; maxiter in 1..%d)", k,
                        kMaxIter);
        if (k > 0 && (q.maxiter != prm->maxiter || q.eo != prm->eo || q.normal != prm->normal ||
                      q.inner_prec != prm->inner_prec || q.inner_recon != prm->inner_recon ||
                      q.reliable_delta != prm->reliable_delta))
            return fail(QCD_ERR_INVALID_ARG,
                        "solve_cg: the systems of one batch may differ in kappa, mu and tol only (system %d)", k);
    }
    if (prm->eo && prm->normal) return fail(QCD_ERR_INVALID_ARG, "solve_cg: normal = 1 needs eo = 0");
    if (prm->inner_prec < QCD_PREC_F64 || prm->inner_prec > QCD_PREC_DF64)
        return fail(QCD_ERR_INVALID_ARG, "solve_cg: bad inner_prec");
    const bool mixed = prm->inner_prec != QCD_PREC_F64;
    if (mixed && prm->inner_recon != 18 && prm->inner_recon != 12 && prm->inner_recon != 8)
        return fail(QCD_ERR_INVALID_ARG, "solve_cg: bad inner_recon");
    if (mixed && !(prm->reliable_delta >= 0.0 && prm->reliable_delta < 1.0))
        return fail(QCD_ERR_INVALID_ARG, "solve_cg: reliable_delta must be 0 (by inner precision) or in (0, 1)");

    const int sp = prm->inner_prec;
    // DF64 links are kept at 18 reals (rebuilding a row in double-float
    // arithmetic costs more than the bytes it saves)
    const int srecon = !mixed ? g->recon : (sp == QCD_PREC_DF64 ? 18 : prm->inner_recon);
    qcd_status st;
    const GaugeView Uh = gauge_view(g, QCD_PREC_F64, g->recon, s, &st);
    if (st != QCD_OK) return st;
    const GaugeView Us = mixed ? gauge_view(g, sp, srecon, s, &st) : Uh;
    if (st != QCD_OK) return st;

    int L = 0;
    while ((1 << L) < nrhs) ++L;
    const int N = 1 << L;
    bool tw = false;
    for (int k = 0; k < nrhs; ++k) tw = tw || prm[k].mu != 0.0;
    OpCtx c{lat, tw, prm->eo != 0, nullptr, nullptr};
    const int nh = c.eo ? 1 : 2;

    // b and x as (batched) full fields
    FieldView bf, xf;
    if (N == 1) {
        bf = view_of(b[0]);
        xf = view_of(x[0]);
    } else {
        bf = ws_field(lat, "cg_bb", 2, QCD_PREC_F64, L);
        xf = ws_field(lat, "cg_xx", 2, QCD_PREC_F64, L);
        if (!bf.hv[0].data || !xf.hv[0].data) return fail(QCD_ERR_OOM, "solve_cg: workspace");
        QCD_TRY(launch_zero(bf, s), "solve_cg: gather");  // padding right-hand sides are zero (solved at once)
        FieldView bv[kMaxRhs];
        for (int k = 0; k < nrhs; ++k) bv[k] = view_of(b[k]);
        QCD_TRY(launch_batch_copy(bf, bv, nrhs, 1, s), "solve_cg: gather");
    }
    // reduction scratch: NV (<= 2) x N partials per block of the largest grid
    Reduction red = reduction_of(lat);
    if (N > 1) {
        const size_t bmax = ((size_t)2 * (lat->h << L) + 63) / 64;
        const size_t need = std::max(red_partials_needed(2 * (size_t)N, bmax), red_partials_needed(N, bmax));
        red.partials = static_cast<double *>(workspace(lat, "cg_partials", need * sizeof(double)));
        red.cap = need;
        if (!red.partials) return fail(QCD_ERR_OOM, "solve_cg: workspace");
    }
    c.red = &red;
    // every kappa/mu-dependent coefficient lives in a device table (one block
    // per rhs; padding rhs repeat system 0), so the cached CG graph depends
    // on neither
    // (the doubles of kMaxRhs blocks, then their float image)
    constexpr size_t kTab = (size_t)kMaxRhs * kCoefPerRhs;
    double *coef = static_cast<double *>(workspace(lat, "cg_coef", kTab * (sizeof(double) + sizeof(float))));
    if (!coef) return fail(QCD_ERR_OOM, "solve_cg: workspace");
    c.coef = coef;
    c.coef_f = reinterpret_cast<const float *>(coef + kTab);
    {
        // staged in the lattice's pinned buffer: the previous solve on this
        // lattice synchronised its stream before returning, so the buffer is free
        static_assert(kTab * 3 / 2 <= (size_t)kCoefHostDoubles, "coefficient staging buffer too small");
        double *table = lat->coef_host;
        float *table_f = reinterpret_cast<float *>(table + kTab);
        for (int k = 0; k < N; ++k) {
            const qcd_solver_params &q = prm[k < nrhs ? k : 0];
            coef_block(table + (size_t)k * kCoefPerRhs, c.eo, q.kappa, 2.0 * q.kappa * q.mu);
        }
        for (size_t j = 0; j < (size_t)N * kCoefPerRhs; ++j) table_f[j] = (float)table[j];
        QCD_TRY(cudaMemcpyAsync(coef, table, (size_t)N * kCoefPerRhs * sizeof(double), cudaMemcpyHostToDevice, s),
                "solve_cg: coefficients");
        QCD_TRY(cudaMemcpyAsync(coef + kTab, table_f, (size_t)N * kCoefPerRhs * sizeof(float), cudaMemcpyHostToDevice, s),
                "solve_cg: coefficients");
    }

    // FP64 fields
    FieldView rhs = c.eo ? ws_field(lat, "cg_rhs", 1, QCD_PREC_F64, L) : bf;
    const FieldView xh = c.eo ? half_of(xf, 0) : xf;
    const FieldView rh = ws_field(lat, "cg_r", nh, QCD_PREC_F64, L);
    const FieldView ph = ws_field(lat, "cg_p", nh, QCD_PREC_F64, L);
    const FieldView qh = ws_field(lat, "cg_q", nh, QCD_PREC_F64, L);
    const FieldView th = ws_field(lat, "cg_t", 1, QCD_PREC_F64, L);
    const FieldView sh = ws_field(lat, "cg_s", nh, QCD_PREC_F64, L);
    if (!rhs.hv[0].data || !rh.hv[0].data || !ph.hv[0].data || !qh.hv[0].data || !th.hv[0].data || !sh.hv[0].data)
        return fail(QCD_ERR_OOM, "solve_cg: workspace");
    // inner fields
    FieldView rs = rh, ps = ph, qs = qh, ts = th, ss = sh, xs = xh;
    if (mixed) {
        rs = ws_field(lat, "cg_rs", nh, sp, L);
        ps = ws_field(lat, "cg_ps", nh, sp, L);
        qs = ws_field(lat, "cg_qs", nh, sp, L);
        ts = ws_field(lat, "cg_ts", 1, sp, L);
        ss = ws_field(lat, "cg_ss", nh, sp, L);
        xs = ws_field(lat, "cg_xs", nh, sp == QCD_PREC_DF64 ? QCD_PREC_DF64 : QCD_PREC_F32, L);
        if (!rs.hv[0].data || !ps.hv[0].data || !qs.hv[0].data || !ts.hv[0].data || !ss.hv[0].data ||
            !xs.hv[0].data)
            return fail(QCD_ERR_OOM, "solve_cg: workspace");
    }

    // ---- right-hand side of the CG system
    FieldView bp{};  // b'_e (eo)
    if (c.eo) {
        const FieldView be = half_of(bf, 0), bo = half_of(bf, 1);
        bp = ws_field(lat, "cg_bp", 1, QCD_PREC_F64, L);
        if (!bp.hv[0].data) return fail(QCD_ERR_OOM, "solve_cg: workspace");
        const FieldView *src = &bo;
        if (tw) {  // th = A^-1 b_o
            const double unused[2][2] = {{1.0, 0.0}, {1.0, 0.0}};
            QCD_TRY(launch_twist(th, bo, unused, s, coef + kCoefTwistInv, kCoefPerRhs), "solve_cg: source");
            src = &th;
        }
        HopArgs h = table_hop(c, kCoefSrcB);  // b' = b_e + kappa D_eo (A^-1 b_o)
        h.fin = FIN_STORE;
        h.out = &bp;
        h.in = src;
        h.y = &be;
        h.out_parity = 0;
        h.twisted = false;  // real coefficients 1 and kappa
        QCD_TRY(hop(lat, Uh, g->recon, h, s), "solve_cg: source");
        HopArgs h3 = table_hop(c, kCoefSrcT);  // th = A^-dag D_oe^dag b'
        h3.fin = FIN_STORE;
        h3.out = &th;
        h3.in = &bp;
        h3.out_parity = 1;
        h3.dagger = 1;
        h3.plain = !tw;
        QCD_TRY(hop(lat, Uh, g->recon, h3, s), "solve_cg: source");
        HopArgs h4 = table_hop(c, kCoefSrcR);  // rhs = A^dag b' - kappa^2 D_eo^dag th
        h4.fin = FIN_STORE;
        h4.out = &rhs;
        h4.in = &th;
        h4.y = &bp;
        h4.out_parity = 0;
        h4.dagger = 1;
        QCD_TRY(hop(lat, Uh, g->recon, h4, s), "solve_cg: source");
    } else if (!prm->normal) {
        rhs = ws_field(lat, "cg_rhs", 2, QCD_PREC_F64, L);
        if (!rhs.hv[0].data) return fail(QCD_ERR_OOM, "solve_cg: workspace");
        QCD_TRY(apply_full_m(c, Uh, g->recon, bf, rhs, 1, s), "solve_cg: source");
    }

    // ---- CG
    const bool split = mixed && (c.eo || !prm->normal);
    const bool mid = split && (sp == QCD_PREC_F16 || sp == QCD_PREC_BF16);
    GaugeView Um = Us;
    FieldView rho_m{}, t_m{}, r_m{};
    if (mid) {
        Um = gauge_view(g, QCD_PREC_F32, srecon, s, &st);
        if (st != QCD_OK) return st;
        rho_m = ws_field(lat, "cg_rho32", nh, QCD_PREC_F32, L);
        t_m = ws_field(lat, "cg_t32", 1, QCD_PREC_F32, L);
        r_m = ws_field(lat, "cg_r32", nh, QCD_PREC_F32, L);
        if (!rho_m.hv[0].data || !t_m.hv[0].data || !r_m.hv[0].data) return fail(QCD_ERR_OOM, "solve_cg: workspace");
    }
    CgFields F{c, Uh, Us, g->recon, srecon, mixed, rhs, xh, rh, qh, th, sh, rs, ps, qs, ts, ss, xs, red, lat->state,
               split, c.eo ? bp : bf, Um, srecon, mid, rho_m, t_m, r_m};
    const double delta = !mixed ? 0.0 : prm->reliable_delta > 0.0 ? prm->reliable_delta : default_reliable_delta(sp);
    RhsValues tol2{};
    for (int k = 0; k < kMaxRhs; ++k) tol2.v[k] = prm[k < nrhs ? k : 0].tol * prm[k < nrhs ? k : 0].tol;
    QCD_TRY(launch_cg_state_init(lat->state, N, tol2, delta * delta, prm->maxiter, s), "solve_cg: init");
    QCD_TRY(launch_cg_setup(rhs, rs, ps, xh, mixed ? &xs : nullptr, F.red, lat->state, s), "solve_cg: setup");

    qcd_status result = QCD_OK;
    if (!profiling_active()) {
        // choose the kernels' launch shapes before they are frozen in the graph
        tuned_tpb(lat, Us, sp, srecon, L, !c.eo, s);
        if (mixed) tuned_tpb(lat, Uh, QCD_PREC_F64, g->recon, L, !c.eo, s);
        cudaGraphExec_t exec = nullptr;
        if (cg_graph(lat, F, &exec) != QCD_OK) {
            // the capture failed (e.g. invalidated by another thread): run
            // the same kernels eagerly instead
            QCD_TRY(cg_eager(lat, F, s), "solve_cg: iterations");
            goto after_loop;
        }
        QCD_TRY(cudaGraphLaunch(exec, s), "solve_cg: graph launch");
        QCD_TRY(read_state(lat, s), "solve_cg: state");
        // kernels the graph ran: per trip the iteration and two control
        // kernels, per reliable update its body
        const int op = c.eo ? 4 : 2;
        const int per_update = split ? (c.eo ? 10 : 7) + (mid ? 1 : 0) : op + 2 + (mixed ? 1 : 0);
        note_launches(lat->state_host->trips * (op + 4) + lat->state_host->reliable_updates * per_update);
    } else {
        QCD_TRY(cg_eager(lat, F, s), "solve_cg: iterations");
    }
after_loop:
    const CgState hs = *lat->state_host;
    if (hs.status == CG_BREAKDOWN)
        result = fail(QCD_ERR_BREAKDOWN, "solve_cg: breakdown (non-positive <p,Ap> or non-finite values)");
    else if (hs.status != CG_DONE)
        result = fail(QCD_ERR_NOT_CONVERGED, "solve_cg: maxiter reached");
    if (mixed && result != QCD_OK) QCD_TRY(launch_cg_accum_x(xh, xs, s), "solve_cg: accumulate");

    // ---- odd sites and residuals
    if (c.eo) {
        const FieldView xo = half_of(xf, 1), bo = half_of(bf, 1);
        HopArgs h = table_hop(c, kCoefRecon);  // x_o = A^-1 b_o + kappa A^-1 D_oe x_e
        h.fin = FIN_STORE;
        h.out = &xo;
        h.in = &xh;
        h.y = &bo;
        h.out_parity = 1;
        QCD_TRY(hop(lat, Uh, g->recon, h, s), "solve_cg: reconstruct");
    }
    double true_rel[kMaxRhs], full_rel[kMaxRhs];
    for (int k = 0; k < N; ++k) true_rel[k] = hs.r[k].b2 > 0 ? std::sqrt(hs.r[k].rr_true / hs.r[k].b2) : 0.0;
    std::vector<double> r2(2 * N);
    if (hs.status != CG_DONE) {  // true residual of the CG system, for the stats
        QCD_TRY(apply_normal(c, Uh, g->recon, xh, qh, th, sh, false, false, s), "solve_cg: residual");
        QCD_TRY(launch_diff_norm2(qh, rhs, F.red, lat->red_out_big, s), "solve_cg: residual");
        QCD_TRY(cudaMemcpyAsync(r2.data(), lat->red_out_big, 2 * N * sizeof(double), cudaMemcpyDeviceToHost, s),
                "solve_cg: residual");
        QCD_TRY(cudaStreamSynchronize(s), "solve_cg: residual");
        for (int k = 0; k < N; ++k) true_rel[k] = r2[N + k] > 0 ? std::sqrt(r2[k] / r2[N + k]) : 0.0;
    }
    // full-system residual |b - M x| / |b|  (normal: |b - M^dag M x| / |b|)
    const FieldView mx = ws_field(lat, "cg_full", 2, QCD_PREC_F64, L);
    if (!mx.hv[0].data) return fail(QCD_ERR_OOM, "solve_cg: workspace");
    QCD_TRY(apply_full_m(c, Uh, g->recon, xf, mx, 0, s), "solve_cg: residual");
    const FieldView *chk = &mx;
    FieldView mx2;
    if (!c.eo && prm->normal) {
        mx2 = ws_field(lat, "cg_full2", 2, QCD_PREC_F64, L);
        if (!mx2.hv[0].data) return fail(QCD_ERR_OOM, "solve_cg: workspace");
        QCD_TRY(apply_full_m(c, Uh, g->recon, mx, mx2, 1, s), "solve_cg: residual");
        chk = &mx2;
    }
    QCD_TRY(launch_diff_norm2(*chk, bf, F.red, lat->red_out_big, s), "solve_cg: residual");
    QCD_TRY(cudaMemcpyAsync(r2.data(), lat->red_out_big, 2 * N * sizeof(double), cudaMemcpyDeviceToHost, s),
            "solve_cg: residual");
    if (N > 1) {
        FieldView xv[kMaxRhs];
        for (int k = 0; k < nrhs; ++k) xv[k] = view_of(x[k]);
        QCD_TRY(launch_batch_copy(xf, xv, nrhs, 0, s), "solve_cg: scatter");
    }
    QCD_TRY(cudaStreamSynchronize(s), "solve_cg: residual");
    for (int k = 0; k < N; ++k) full_rel[k] = r2[N + k] > 0 ? std::sqrt(r2[k] / r2[N + k]) : 0.0;

    if (stats) {
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int k = 0; k < nrhs; ++k) {
            stats[k].iterations = hs.r[k].status == CG_DONE ? hs.r[k].iter_done : hs.iter;
            stats[k].reliable_updates = hs.reliable_updates;
            stats[k].true_rel_residual = true_rel[k];
            stats[k].full_rel_residual = full_rel[k];
            stats[k].seconds = secs;
        }
    }
    return result;
}

extern "C" qcd_status qcd_solve_cg(const qcd_gauge *g, qcd_spinor *x, const qcd_spinor *b,
                                   const qcd_solver_params *prm, qcd_solver_stats *stats, void *stream)
{
    qcd_spinor *xs[1] = {x};
    const qcd_spinor *bs[1] = {b};
    return solve_impl(g, xs, bs, 1, prm, stats, static_cast<cudaStream_t>(stream), nullptr);
}

extern "C" qcd_status qcd_solve_cg_multi(const qcd_gauge *g, qcd_spinor *const *x, const qcd_spinor *const *b,
                                         int nrhs, const qcd_solver_params *prm, qcd_solver_stats *stats,
                                         void *stream)
{
    if (!prm) return fail(QCD_ERR_INVALID_ARG, "solve_cg_multi: NULL argument");
    if (nrhs < 1 || nrhs > kMaxRhs) return fail(QCD_ERR_INVALID_ARG, "solve_cg_multi: nrhs = %d not in 1..%d", nrhs, kMaxRhs);
    std::vector<qcd_solver_params> p((size_t)nrhs, *prm);
    return solve_impl(g, x, b, nrhs, p.data(), stats, static_cast<cudaStream_t>(stream), nullptr);
}

extern "C" qcd_status qcd_solve_cg_batch(const qcd_gauge *g, qcd_spinor *const *x, const qcd_spinor *const *b, int n,
                                         const qcd_solver_params *prm, qcd_solver_stats *stats, void *stream)
{
    return solve_impl(g, x, b, n, prm, stats, static_cast<cudaStream_t>(stream), nullptr);
}
