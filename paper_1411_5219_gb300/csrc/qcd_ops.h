// Host-side launchers of the libqcd kernels (internal).
#pragma once

#include "qcd_internal.cuh"

namespace qcd {

// Counts kernel launches (qcd_kernel_launches).
void note_launches(int n = 1);

// A spinor field made of one (half) or two (full: even, odd) half fields of
// h sites each, in storage precision `prec`.
struct FieldView {
    SpinorView hv[2];
    int nh;        // 1 or 2
    int h;         // elements per half: sites << rhs_log2
    int prec;      // qcd_prec
    int rhs_log2;  // batched field: element = site * 2^rhs_log2 + rhs
};

// out = c[chi] * in (one complex factor per chirality), e.g. A^-1 psi.
// out = c[chirality] in; with `table`, rhs r takes its c from table + r * stride (4 doubles).
cudaError_t launch_twist(const FieldView &out, const FieldView &in, const double c[2][2], cudaStream_t s,
                         const double *table = nullptr, int stride = 0);
// dst = src with precision conversion.
cudaError_t launch_convert(const FieldView &dst, const FieldView &src, cudaStream_t s);
cudaError_t launch_zero(const FieldView &f, cudaStream_t s);
// |f|^2 reduced in FP64; `fin` says what the last block does with it.
cudaError_t launch_norm2(const FieldView &f, const Reduction &red, FinalizeKind fin, CgState *st, double *out,
                         cudaStream_t s);
// Per rhs r of the batched F64 fields: out[r] = |a - b|^2, out[n + r] = |b|^2.
cudaError_t launch_diff_norm2(const FieldView &a, const FieldView &b, const Reduction &red, double *out,
                              cudaStream_t s);

// CG vector steps.  The CG state lives on the device; every kernel below
// except cg_true_residual returns at once unless state->status is RUNNING.
// One double per right-hand side (kernel parameter).
struct RhsValues {
    double v[kMaxRhs];
};
cudaError_t launch_cg_state_init(CgState *st, int nrhs, const RhsValues &tol2, double delta2, int maxiter,
                                 cudaStream_t s);
// r = rhs (cast), p = r, x = 0, xs = 0 (if given); rr = |rhs|^2; status.
cudaError_t launch_cg_setup(const FieldView &rhs, const FieldView &r, const FieldView &p, const FieldView &x,
                            const FieldView *xs, const Reduction &red, CgState *st, cudaStream_t s);
// x += alpha p, r -= alpha q, |r|^2 -> beta / status.  x is F64 (plain) or
// F32 (mixed), p, r, q share one precision.
cudaError_t launch_cg_xr(const FieldView &x, const FieldView &p, const FieldView &r, const FieldView &q,
                         const Reduction &red, CgState *st, cudaStream_t s);
// p = r + beta p
cudaError_t launch_cg_p(const FieldView &p, const FieldView &r, CgState *st, cudaStream_t s);
// xhi += xs, xs = 0 (mixed precision, before a reliable update)
cudaError_t launch_cg_accum_x(const FieldView &xhi, const FieldView &xs, cudaStream_t s);
// rho = rhs0 - q (F64 defect of the un-normalised system) and rs = cast(rho).
cudaError_t launch_cg_defect(const FieldView &rhs0, const FieldView &q, const FieldView &rho, const FieldView &rs,
                             cudaStream_t s);
// |f|^2 (F64) -> FIN_CG_TRUE, only while the CG state is CG_VERIFY.
cudaError_t launch_cg_verify(const FieldView &f, const Reduction &red, CgState *st, cudaStream_t s);
// rhi = rhs - q (F64), |rhi|^2 -> reliable-update decision; rs = cast(rhi) if given.
cudaError_t launch_cg_true_residual(const FieldView &rhs, const FieldView &q, const FieldView &rhi,
                                   const FieldView *rs, const Reduction &red, CgState *st, cudaStream_t s);


// Graph control kernels (cudaGraphSetConditional on the loop / reliable-update handles).
cudaError_t launch_cg_ctrl_reliable(const CgState *st, cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t launch_cg_ctrl_loop(CgState *st, cudaGraphConditionalHandle h, cudaStream_t s);

// Copy between rhs 0..n-1 of a batched field and n plain fields of the same
// precision and halves, in one launch: to_batch = 1 copies plain[k] ->
// batched[rhs k] (other rhs untouched).
struct PlainSet {
    FieldView f[kMaxRhs];
};
cudaError_t launch_batch_copy(const FieldView &batched, const FieldView *plain, int n, int to_batch, cudaStream_t s);

// Staggered hopping term (csrc/staggered.cu).  in/out indexed by output
// parity as for DslashLaunch; staggered fields hold 3 complex per site.
struct KsLaunch {
    Geom g;
    int out_parity;
    int both;
    GaugeView U;
    SpinorView in[2], out[2];
};
cudaError_t launch_dslash_ks(int prec, int recon, const KsLaunch &a, cudaStream_t s);
cudaError_t launch_ks_pack(const FieldView &f, int parity, const double2 *aos, const Geom &g, cudaStream_t s);
cudaError_t launch_ks_unpack(double2 *aos, const FieldView &f, int parity, const Geom &g, cudaStream_t s);

// Layout conversion between the host AoS form (FP64, lexicographic) and the
// device SoA form.
cudaError_t launch_gauge_pack(const GaugeView &dst, int prec, int recon, const double2 *aos, const Geom &g,
                              cudaStream_t s);
cudaError_t launch_gauge_convert(const GaugeView &dst, int dprec, int drecon, const GaugeView &src, int sprec,
                                 int srecon, const Geom &g, cudaStream_t s);
cudaError_t gauge_recon8_error(const GaugeView &dst, int prec, const double2 *aos, const GaugeView &src, int sprec,
                               int srecon, const Geom &g, cudaStream_t s, double *max_err);
// parity: 0/1 for a half field in parity-compacted host layout, 2 for a
// full field in lexicographic host layout.
cudaError_t launch_spinor_pack(const FieldView &dst, int parity, const double2 *aos, const Geom &g, cudaStream_t s);
cudaError_t launch_spinor_unpack(double2 *aos, const FieldView &src, int parity, const Geom &g, cudaStream_t s);

}  // namespace qcd
