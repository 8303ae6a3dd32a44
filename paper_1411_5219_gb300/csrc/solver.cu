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

#include "qcd_handles.h"

namespace qcd {
namespace {

struct OpCtx {
    const qcd_lattice *lat;
    double kappa, a;  // a = 2 kappa mu
    bool eo;
};

// out = Mhat^dag Mhat in (eo) or M^dag M in (full).  t (odd half) and s
// (even half, or full) are temporaries of the same precision.  With
// reduce_alpha the second kernel also reduces |Mhat in|^2 into alpha.
cudaError_t apply_normal(const OpCtx &c, const GaugeView &U, int recon, const FieldView &in, const FieldView &out,
                         const FieldView &t, const FieldView &s, bool reduce_alpha, bool check, cudaStream_t st)
{
    const bool tw = c.a != 0.0;
    cudaError_t e;
    if (c.eo) {
        HopArgs h{};
        h.check_status = check;
        h.fin = FIN_CG_ALPHA;
        // t = A^-1 D_oe in
        h.out = &t;
        h.in = &in;
        h.out_parity = 1;
        h.plain = !tw;
        h.twisted = tw;
        h.cd = coef_twist_inv(c.a);
        if ((e = hop(c.lat, U, recon, h, st)) != cudaSuccess) return e;
        // s = A in - kappa^2 D_eo t   (|s|^2 -> alpha)
        HopArgs h2{};
        h2.check_status = check;
        h2.fin = FIN_CG_ALPHA;
        h2.out = &s;
        h2.in = &t;
        h2.y = &in;
        h2.out_parity = 0;
        h2.twisted = tw;
        h2.cy = coef_twist(c.a);
        h2.cd = coef_real(-c.kappa * c.kappa);
        h2.reduce = reduce_alpha;
        if ((e = hop(c.lat, U, recon, h2, st)) != cudaSuccess) return e;
        // t = A^-dag D_oe^dag s
        HopArgs h3 = h;
        h3.in = &s;
        h3.dagger = 1;
        h3.cd = coef_twist_inv(-c.a);
        if ((e = hop(c.lat, U, recon, h3, st)) != cudaSuccess) return e;
        // out = A^dag s - kappa^2 D_eo^dag t
        HopArgs h4 = h2;
        h4.out = &out;
        h4.in = &t;
        h4.y = &s;
        h4.dagger = 1;
        h4.cy = coef_twist(-c.a);
        h4.reduce = false;
        return hop(c.lat, U, recon, h4, st);
    }
    // s = M in = A in - kappa D in  (|s|^2 -> alpha)
    HopArgs h{};
    h.check_status = check;
    h.fin = FIN_CG_ALPHA;
    h.out = &s;
    h.in = &in;
    h.y = &in;
    h.both = true;
    h.twisted = tw;
    h.cy = coef_twist(c.a);
    h.cd = coef_real(-c.kappa);
    h.reduce = reduce_alpha;
    if ((e = hop(c.lat, U, recon, h, st)) != cudaSuccess) return e;
    // out = M^dag s
    HopArgs h2 = h;
    h2.out = &out;
    h2.in = &s;
    h2.y = &s;
    h2.dagger = 1;
    h2.cy = coef_twist(-c.a);
    h2.reduce = false;
    return hop(c.lat, U, recon, h2, st);
}

// out = M in on a full field (dagger: M^dag).
cudaError_t apply_full_m(const OpCtx &c, const GaugeView &U, int recon, const FieldView &in, const FieldView &out,
                         int dagger, cudaStream_t st)
{
    HopArgs h{};
    h.fin = FIN_STORE;
    h.out = &out;
    h.in = &in;
    h.y = &in;
    h.both = true;
    h.dagger = dagger;
    h.twisted = c.a != 0.0;
    h.cy = coef_twist(dagger ? -c.a : c.a);
    h.cd = coef_real(-c.kappa);
    return hop(c.lat, U, recon, h, st);
}

}  // namespace
}  // namespace qcd

using namespace qcd;

#define QCD_TRY(expr, what)                                   \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return check_cuda(e_, what);   \
    } while (0)

extern "C" qcd_status qcd_solve_cg(const qcd_gauge *g, qcd_spinor *x, const qcd_spinor *b,
                                   const qcd_solver_params *prm, qcd_solver_stats *stats, void *stream)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (!g || !x || !b || !prm) return fail(QCD_ERR_INVALID_ARG, "solve_cg: NULL argument");
    const qcd_lattice *lat = g->lat;
    if (x->lat != lat || b->lat != lat) return fail(QCD_ERR_INVALID_ARG, "solve_cg: lattices differ");
    if (x->parity != QCD_PARITY_FULL || b->parity != QCD_PARITY_FULL || x->prec != QCD_PREC_F64 ||
        b->prec != QCD_PREC_F64)
        return fail(QCD_ERR_INVALID_ARG, "solve_cg: x and b must be FULL F64 fields");
    if (x == b || x->data == b->data) return fail(QCD_ERR_INVALID_ARG, "solve_cg: x aliases b");
    if (g->prec != QCD_PREC_F64) return fail(QCD_ERR_INVALID_ARG, "solve_cg: the gauge field must be F64");
    if (!(prm->tol > 0.0) || prm->maxiter < 1 || !std::isfinite(prm->kappa) || !std::isfinite(prm->mu))
        return fail(QCD_ERR_INVALID_ARG, "solve_cg: bad tol/maxiter/kappa/mu");
    if (prm->eo && prm->normal) return fail(QCD_ERR_INVALID_ARG, "solve_cg: normal = 1 needs eo = 0");
    if (prm->inner_prec < QCD_PREC_F64 || prm->inner_prec > QCD_PREC_BF16)
        return fail(QCD_ERR_INVALID_ARG, "solve_cg: bad inner_prec");
    const bool mixed = prm->inner_prec != QCD_PREC_F64;
    if (mixed && prm->inner_recon != 18 && prm->inner_recon != 12)
        return fail(QCD_ERR_INVALID_ARG, "solve_cg: bad inner_recon");
    if (mixed && !(prm->reliable_delta > 0.0 && prm->reliable_delta < 1.0))
        return fail(QCD_ERR_INVALID_ARG, "solve_cg: reliable_delta must be in (0, 1)");

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int sp = prm->inner_prec;
    const int srecon = mixed ? prm->inner_recon : g->recon;
    qcd_status st;
    const GaugeView Uh = gauge_view(g, QCD_PREC_F64, g->recon, s, &st);
    if (st != QCD_OK) return st;
    const GaugeView Us = mixed ? gauge_view(g, sp, srecon, s, &st) : Uh;
    if (st != QCD_OK) return st;

    OpCtx c{lat, prm->kappa, 2.0 * prm->kappa * prm->mu, prm->eo != 0};
    const bool tw = c.a != 0.0;
    const int nh = c.eo ? 1 : 2;
    const FieldView bf = view_of(b), xf = view_of(x);

    // FP64 fields
    FieldView rhs = c.eo ? ws_field(lat, "cg_rhs", 1, QCD_PREC_F64) : bf;
    const FieldView xh = c.eo ? view_half(x, 0) : xf;
    const FieldView rh = ws_field(lat, "cg_r", nh, QCD_PREC_F64);
    const FieldView ph = ws_field(lat, "cg_p", nh, QCD_PREC_F64);
    const FieldView qh = ws_field(lat, "cg_q", nh, QCD_PREC_F64);
    const FieldView th = ws_field(lat, "cg_t", 1, QCD_PREC_F64);
    const FieldView sh = ws_field(lat, "cg_s", nh, QCD_PREC_F64);
    if (!rhs.hv[0].data || !rh.hv[0].data || !ph.hv[0].data || !qh.hv[0].data || !th.hv[0].data || !sh.hv[0].data)
        return fail(QCD_ERR_OOM, "solve_cg: workspace");
    // inner fields
    FieldView rs = rh, ps = ph, qs = qh, ts = th, ss = sh, xs = xh;
    if (mixed) {
        rs = ws_field(lat, "cg_rs", nh, sp);
        ps = ws_field(lat, "cg_ps", nh, sp);
        qs = ws_field(lat, "cg_qs", nh, sp);
        ts = ws_field(lat, "cg_ts", 1, sp);
        ss = ws_field(lat, "cg_ss", nh, sp);
        xs = ws_field(lat, "cg_xs", nh, QCD_PREC_F32);
        if (!rs.hv[0].data || !ps.hv[0].data || !qs.hv[0].data || !ts.hv[0].data || !ss.hv[0].data ||
            !xs.hv[0].data)
            return fail(QCD_ERR_OOM, "solve_cg: workspace");
    }

    // ---- right-hand side of the CG system
    if (c.eo) {
        const FieldView be = view_half(b, 0), bo = view_half(b, 1);
        const FieldView bp = ws_field(lat, "cg_bp", 1, QCD_PREC_F64);
        if (!bp.hv[0].data) return fail(QCD_ERR_OOM, "solve_cg: workspace");
        const FieldView *src = &bo;
        if (tw) {  // th = A^-1 b_o
            const Coef ci = coef_twist_inv(c.a);
            QCD_TRY(launch_twist(th, bo, ci.c, s), "solve_cg: source");
            src = &th;
        }
        HopArgs h{};  // b' = b_e + kappa D_eo (A^-1 b_o)
        h.fin = FIN_STORE;
        h.out = &bp;
        h.in = src;
        h.y = &be;
        h.out_parity = 0;
        h.cy = coef_real(1.0);
        h.cd = coef_real(c.kappa);
        QCD_TRY(hop(lat, Uh, g->recon, h, s), "solve_cg: source");
        HopArgs h3{};  // th = A^-dag D_oe^dag b'
        h3.fin = FIN_STORE;
        h3.out = &th;
        h3.in = &bp;
        h3.out_parity = 1;
        h3.dagger = 1;
        h3.plain = !tw;
        h3.twisted = tw;
        h3.cd = coef_twist_inv(-c.a);
        QCD_TRY(hop(lat, Uh, g->recon, h3, s), "solve_cg: source");
        HopArgs h4{};  // rhs = A^dag b' - kappa^2 D_eo^dag th
        h4.fin = FIN_STORE;
        h4.out = &rhs;
        h4.in = &th;
        h4.y = &bp;
        h4.out_parity = 0;
        h4.dagger = 1;
        h4.twisted = tw;
        h4.cy = coef_twist(-c.a);
        h4.cd = coef_real(-c.kappa * c.kappa);
        QCD_TRY(hop(lat, Uh, g->recon, h4, s), "solve_cg: source");
    } else if (!prm->normal) {
        rhs = ws_field(lat, "cg_rhs", 2, QCD_PREC_F64);
        if (!rhs.hv[0].data) return fail(QCD_ERR_OOM, "solve_cg: workspace");
        QCD_TRY(apply_full_m(c, Uh, g->recon, bf, rhs, 1, s), "solve_cg: source");
    }

    // ---- CG
    const Reduction red = reduction_of(lat);
    const double delta = mixed ? prm->reliable_delta : 0.0;
    QCD_TRY(launch_cg_state_init(lat->state, prm->tol * prm->tol, delta * delta, prm->maxiter, s), "solve_cg: init");
    QCD_TRY(launch_cg_setup(rhs, rs, ps, xh, mixed ? &xs : nullptr, red, lat->state, s), "solve_cg: setup");

    auto read_state = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(lat->state_host, lat->state, sizeof(CgState), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e;
    };
    auto true_residual = [&]() -> cudaError_t {
        cudaError_t e = cudaSuccess;
        if (mixed) e = launch_cg_accum_x(xh, xs, s);
        if (e == cudaSuccess) e = apply_normal(c, Uh, g->recon, xh, qh, th, sh, false, false, s);
        if (e == cudaSuccess) e = launch_cg_true_residual(rhs, qh, rh, mixed ? &rs : nullptr, red, lat->state, s);
        if (e == cudaSuccess) e = launch_cg_p(ps, rs, lat->state, s);
        return e;
    };

    QCD_TRY(read_state(), "solve_cg: state");
    int batch = 2;
    double last_rr = lat->state_host->rr;
    int last_iter = 0;
    qcd_status result = QCD_OK;
    for (;;) {
        const int status = lat->state_host->status;
        if (status == CG_DONE) break;
        if (status == CG_BREAKDOWN) {
            result = fail(QCD_ERR_BREAKDOWN, "solve_cg: breakdown (non-positive <p,Ap> or non-finite values)");
            break;
        }
        if (status == CG_MAXITER) {
            result = fail(QCD_ERR_NOT_CONVERGED, "solve_cg: maxiter reached");
            break;
        }
        if (status == CG_CONVERGED || status == CG_RELIABLE) {
            QCD_TRY(true_residual(), "solve_cg: true residual");
        }
        for (int k = 0; k < batch; ++k) {
            QCD_TRY(apply_normal(c, Us, srecon, ps, qs, ts, ss, true, true, s), "solve_cg: operator");
            QCD_TRY(launch_cg_xr(mixed ? xs : xh, ps, rs, qs, red, lat->state, s), "solve_cg: update");
            QCD_TRY(launch_cg_p(ps, rs, lat->state, s), "solve_cg: update");
        }
        QCD_TRY(read_state(), "solve_cg: state");
        // Size the next batch from the observed convergence rate.
        const CgState &hs = *lat->state_host;
        const int done = hs.iter - last_iter;
        if (done > 0 && hs.rr > 0.0 && last_rr > hs.rr && hs.status == CG_RUNNING) {
            const double rate = std::log(last_rr / hs.rr) / done;
            const double rem = std::log(hs.rr / hs.rr_stop) / rate;
            batch = (int)std::min(64.0, std::max(2.0, 0.9 * rem));
        } else {
            batch = std::min(64, batch * 2);
        }
        last_rr = hs.rr;
        last_iter = hs.iter;
    }
    if (mixed && result != QCD_OK) QCD_TRY(launch_cg_accum_x(xh, xs, s), "solve_cg: accumulate");

    // ---- odd sites and residuals
    const CgState hs = *lat->state_host;
    double true_rel = std::sqrt(hs.b2 > 0 ? hs.rr_true / hs.b2 : 0.0);
    if (c.eo) {
        const FieldView xo = view_half(x, 1), bo = view_half(b, 1);
        HopArgs h{};  // x_o = A^-1 b_o + kappa A^-1 D_oe x_e
        h.fin = FIN_STORE;
        h.out = &xo;
        h.in = &xh;
        h.y = &bo;
        h.out_parity = 1;
        h.twisted = tw;
        h.cy = coef_twist_inv(c.a);
        h.cd = coef_scale(coef_twist_inv(c.a), c.kappa);
        QCD_TRY(hop(lat, Uh, g->recon, h, s), "solve_cg: reconstruct");
    }
    if (hs.status != CG_DONE) {  // true residual of the CG system, for the stats
        QCD_TRY(apply_normal(c, Uh, g->recon, xh, qh, th, sh, false, false, s), "solve_cg: residual");
        QCD_TRY(launch_diff_norm2(qh, rhs, red, lat->red_out, s), "solve_cg: residual");
        double r2[2];
        QCD_TRY(cudaMemcpyAsync(r2, lat->red_out, sizeof(r2), cudaMemcpyDeviceToHost, s), "solve_cg: residual");
        QCD_TRY(cudaStreamSynchronize(s), "solve_cg: residual");
        true_rel = r2[1] > 0 ? std::sqrt(r2[0] / r2[1]) : 0.0;
    }
    // full-system residual |b - M x| / |b|  (normal: |b - M^dag M x| / |b|)
    const FieldView mx = ws_field(lat, "cg_full", 2, QCD_PREC_F64);
    if (!mx.hv[0].data) return fail(QCD_ERR_OOM, "solve_cg: workspace");
    QCD_TRY(apply_full_m(c, Uh, g->recon, xf, mx, 0, s), "solve_cg: residual");
    const FieldView *chk = &mx;
    FieldView mx2;
    if (!c.eo && prm->normal) {
        mx2 = ws_field(lat, "cg_full2", 2, QCD_PREC_F64);
        if (!mx2.hv[0].data) return fail(QCD_ERR_OOM, "solve_cg: workspace");
        QCD_TRY(apply_full_m(c, Uh, g->recon, mx, mx2, 1, s), "solve_cg: residual");
        chk = &mx2;
    }
    QCD_TRY(launch_diff_norm2(*chk, bf, red, lat->red_out, s), "solve_cg: residual");
    double r2[2];
    QCD_TRY(cudaMemcpyAsync(r2, lat->red_out, sizeof(r2), cudaMemcpyDeviceToHost, s), "solve_cg: residual");
    QCD_TRY(cudaStreamSynchronize(s), "solve_cg: residual");

    if (stats) {
        stats->iterations = hs.iter;
        stats->reliable_updates = hs.reliable_updates;
        stats->true_rel_residual = true_rel;
        stats->full_rel_residual = r2[1] > 0 ? std::sqrt(r2[0] / r2[1]) : 0.0;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return result;
}
