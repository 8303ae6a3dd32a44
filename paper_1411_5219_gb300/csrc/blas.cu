// Vector kernels of the CG solver and field utilities: precision
// conversion, chiral twist, norms, and the fused CG updates
// (x += alpha p, r -= alpha q, |r|^2), (p = r + beta p) and the FP64
// true residual of a reliable update.  The paper's physics package offers
// such "algebraic operations like saxpy" next to the fermion matrices
// (CL2QCD, arXiv:1411.5219, Sec. 4); here each one is a single pass over
// the fields with FP64 reductions of fixed summation order.
#include "qcd_ops.h"

namespace qcd {

namespace {

template <typename SF>
__device__ __forceinline__ Spinor<typename SF::R> ld(const FieldView &f, int k)
{
    const int hh = k >= f.h;
    return SF::load(f.hv[hh], k - hh * f.h);
}
template <typename SF>
__device__ __forceinline__ void st(const FieldView &f, int k, const Spinor<typename SF::R> &v)
{
    const int hh = k >= f.h;
    SF::store(f.hv[hh], k - hh * f.h, v);
}

template <typename R2, typename R1>
__device__ __forceinline__ Spinor<R2> cvt(const Spinor<R1> &a)
{
    Spinor<R2> b;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) b.c[s][c] = mk((R2)a.c[s][c].re, (R2)a.c[s][c].im);
    return b;
}

template <typename R>
__device__ __forceinline__ R norm2(const Spinor<R> &a)
{
    R n = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) n += a.c[s][c].re * a.c[s][c].re + a.c[s][c].im * a.c[s][c].im;
    return n;
}

template <typename R>
__device__ __forceinline__ Spinor<R> zero_spinor()
{
    Spinor<R> z;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) z.c[s][c] = mk((R)0, (R)0);
    return z;
}

__host__ __device__ inline int nsites(const FieldView &f) { return f.nh * f.h; }

// ---------------------------------------------------------------- kernels

template <typename SO, typename SI>
__global__ void __launch_bounds__(kThreads) convert_kernel(const FieldView out, const FieldView in)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nsites(out)) st<SO>(out, k, cvt<typename SO::R>(ld<SI>(in, k)));
}

template <typename SF>
__global__ void __launch_bounds__(kThreads) zero_kernel(const FieldView f)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nsites(f)) st<SF>(f, k, zero_spinor<typename SF::R>());
}

template <typename SF>
__global__ void __launch_bounds__(kThreads) twist_kernel(const FieldView out, const FieldView in, const double cr0,
                                                         const double ci0, const double cr1, const double ci1,
                                                         const double *table, const int stride)
{
    using R = typename SF::R;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsites(out)) return;
    cx<R> c[2] = {mk((R)cr0, (R)ci0), mk((R)cr1, (R)ci1)};
    if (table) {  // per-rhs coefficients
        const double *t = table + (size_t)(k & ((1 << out.rhs_log2) - 1)) * stride;
        c[0] = mk((R)t[0], (R)t[1]);
        c[1] = mk((R)t[2], (R)t[3]);
    }
    Spinor<R> a = ld<SF>(in, k);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) a.c[s][cc] = cmul(c[s >> 1], a.c[s][cc]);
    st<SF>(out, k, a);
}

template <typename SF>
__global__ void __launch_bounds__(kThreads) norm2_kernel(const FieldView f, const Reduction red, const FinalizeKind fin,
                                                         CgState *stt, double *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (k < nsites(f)) v[0] = (double)norm2(ld<SF>(f, k));
    grid_reduce_rhs<1>(v, f.rhs_log2, red, fin, stt, out);
}

__global__ void __launch_bounds__(kThreads) diff_norm2_kernel(const FieldView a, const FieldView b, const Reduction red,
                                                              double *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (k < nsites(a)) {
        const Spinor<double> x = ld<SpF64>(a, k), y = ld<SpF64>(b, k);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double dr = x.c[s][c].re - y.c[s][c].re, di = x.c[s][c].im - y.c[s][c].im;
                v[0] += dr * dr + di * di;
                v[1] += y.c[s][c].re * y.c[s][c].re + y.c[s][c].im * y.c[s][c].im;
            }
    }
    grid_reduce_rhs<2>(v, a.rhs_log2, red, FIN_STORE, nullptr, out);
}

__global__ void cg_state_init_kernel(CgState *s, int nrhs, const RhsValues tol2, double delta2, int maxiter)
{
    for (int k = 0; k < kMaxRhs; ++k) {
        CgRhs &q = s->r[k];
        q.rr = q.rr_prev = q.pAp = q.alpha = q.beta = 0.0;
        q.rr_stop = q.rr_max = q.rr_true = q.b2 = 0.0;
        q.tol2 = tol2.v[k];
        q.status = CG_DONE;
        q.iter_done = 0;
    }
    s->nrhs = nrhs;
    s->tol2 = tol2.v[0];
    s->delta2 = delta2;
    s->iter = 0;
    s->maxiter = maxiter;
    s->status = CG_RUNNING;
    s->reliable_updates = 0;
    s->trips = 0;
    s->trip_limit = maxiter + 64;
}


// Graph control: run the reliable-update body when the iteration asked for it.
__global__ void cg_ctrl_reliable_kernel(const CgState *st, cudaGraphConditionalHandle h)
{
    const int s = st->status;
    cudaGraphSetConditional(h, (s == CG_RELIABLE || s == CG_CONVERGED) ? 1u : 0u);
}

// Graph control: repeat the loop body while CG runs; the trip cap bounds the
// loop whatever the state holds.
__global__ void cg_ctrl_loop_kernel(CgState *st, cudaGraphConditionalHandle h)
{
    st->trips += 1;
    const bool go = st->status == CG_RUNNING && st->iter < st->maxiter && st->trips < st->trip_limit;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// r = rhs, p = r (both in the CG precision), x = 0, xs = 0; |rhs|^2.
template <typename SR, typename SX, typename SS>
__global__ void __launch_bounds__(kThreads) cg_setup_kernel(const FieldView rhs, const FieldView r, const FieldView p,
                                                            const FieldView x, const FieldView xs, const bool has_xs,
                                                            const Reduction red, CgState *stt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (k < nsites(rhs)) {
        const Spinor<double> b = ld<SpF64>(rhs, k);
        const Spinor<typename SR::R> bc = cvt<typename SR::R>(b);
        st<SR>(r, k, bc);
        st<SR>(p, k, bc);
        st<SX>(x, k, zero_spinor<typename SX::R>());
        if (has_xs) st<SS>(xs, k, zero_spinor<typename SS::R>());
        v[0] = norm2(b);
    }
    grid_reduce_rhs<1>(v, rhs.rhs_log2, red, FIN_CG_INIT, stt, nullptr);
}

// x += alpha p; r -= alpha q; |r|^2.
template <typename SX, typename SF>
__global__ void __launch_bounds__(kThreads) cg_xr_kernel(const FieldView x, const FieldView p, const FieldView r,
                                                         const FieldView q, const Reduction red, CgState *stt)
{
    if (stt->status != CG_RUNNING) return;
    using R = typename SF::R;
    using RX = typename SX::R;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    using RedT = typename std::conditional<std::is_same<R, float>::value, float, double>::type;
    RedT v[1] = {RedT(0)};
    if (k < nsites(x)) {
        const double alpha = stt->r[k & ((1 << x.rhs_log2) - 1)].alpha;
        const Spinor<R> pp = ld<SF>(p, k), qq = ld<SF>(q, k);
        Spinor<R> rr = ld<SF>(r, k);
        Spinor<RX> xx = ld<SX>(x, k);
        const RX ax = (RX)alpha;
        const R ar = (R)alpha;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xx.c[s][c].re = fma(ax, (RX)pp.c[s][c].re, xx.c[s][c].re);
                xx.c[s][c].im = fma(ax, (RX)pp.c[s][c].im, xx.c[s][c].im);
                rr.c[s][c].re = fma(-ar, qq.c[s][c].re, rr.c[s][c].re);
                rr.c[s][c].im = fma(-ar, qq.c[s][c].im, rr.c[s][c].im);
            }
        st<SX>(x, k, xx);
        st<SF>(r, k, rr);
        v[0] = (RedT)norm2(rr);
    }
    grid_reduce_rhs<1>(v, x.rhs_log2, red, FIN_CG_RR, stt, nullptr);
}

// p = r + beta p
template <typename SF>
__global__ void __launch_bounds__(kThreads) cg_p_kernel(const FieldView p, const FieldView r, const CgState *stt)
{
    if (stt->status != CG_RUNNING) return;
    using R = typename SF::R;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsites(p)) return;
    const R beta = (R)stt->r[k & ((1 << p.rhs_log2) - 1)].beta;
    Spinor<R> pp = ld<SF>(p, k);
    const Spinor<R> rr = ld<SF>(r, k);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pp.c[s][c].re = fma(beta, pp.c[s][c].re, rr.c[s][c].re);
            pp.c[s][c].im = fma(beta, pp.c[s][c].im, rr.c[s][c].im);
        }
    st<SF>(p, k, pp);
}

// xhi += xs; xs = 0
template <typename SS>
__global__ void __launch_bounds__(kThreads) cg_accum_x_kernel(const FieldView xhi, const FieldView xs)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsites(xhi)) return;
    Spinor<double> a = ld<SpF64>(xhi, k);
    const Spinor<double> b = cvt<double>(ld<SS>(xs, k));
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) a.c[s][c] = a.c[s][c] + b.c[s][c];
    st<SpF64>(xhi, k, a);
    st<SS>(xs, k, zero_spinor<typename SS::R>());
}

// rhi = rhs - q; |rhi|^2; rs = cast(rhi)
template <typename SS>
__global__ void __launch_bounds__(kThreads) cg_true_residual_kernel(const FieldView rhs, const FieldView q,
                                                                    const FieldView rhi, const FieldView rs,
                                                                    const bool has_rs, const Reduction red,
                                                                    CgState *stt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (k < nsites(rhs)) {
        Spinor<double> a = ld<SpF64>(rhs, k);
        const Spinor<double> b = ld<SpF64>(q, k);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) a.c[s][c] = a.c[s][c] - b.c[s][c];
        st<SpF64>(rhi, k, a);
        if (has_rs) st<SS>(rs, k, cvt<typename SS::R>(a));
        v[0] = norm2(a);
    }
    grid_reduce_rhs<1>(v, rhs.rhs_log2, red, FIN_CG_TRUE, stt, nullptr);
}

// rho = rhs0 - q (FP64 defect of the un-normalised system), rs = cast(rho)
template <typename SS>
__global__ void __launch_bounds__(kThreads) cg_defect_kernel(const FieldView rhs0, const FieldView q,
                                                             const FieldView rho, const FieldView rs)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsites(rhs0)) return;
    Spinor<double> a = ld<SpF64>(rhs0, k);
    const Spinor<double> b = ld<SpF64>(q, k);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) a.c[s][c] = a.c[s][c] - b.c[s][c];
    st<SpF64>(rho, k, a);
    st<SS>(rs, k, cvt<typename SS::R>(a));
}

// |f|^2 per rhs (FP64) -> FIN_CG_TRUE, only while the state is CG_VERIFY
__global__ void __launch_bounds__(kThreads) cg_verify_kernel(const FieldView f, const Reduction red, CgState *stt)
{
    if (stt->status != CG_VERIFY) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (k < nsites(f)) v[0] = norm2(ld<SpF64>(f, k));
    grid_reduce_rhs<1>(v, f.rhs_log2, red, FIN_CG_TRUE, stt, nullptr);
}

// batched[(i << L) | rhs] <-> plain[rhs][i] for rhs < n, over both halves,
// one thread per batched element: a warp reads (or writes) consecutive
// batched elements, and the same few sites of each plain field.
template <typename SF>
__global__ void __launch_bounds__(kThreads) batch_copy_kernel(const FieldView b, const PlainSet pl, const int n,
                                                              const int to_batch)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsites(b)) return;
    const int hh = k >= b.h, e = k - hh * b.h;
    const int rhs = e & ((1 << b.rhs_log2) - 1), i = e >> b.rhs_log2;
    if (rhs >= n) return;
    if (to_batch)
        SF::store(b.hv[hh], e, SF::load(pl.f[rhs].hv[hh], i));
    else
        SF::store(pl.f[rhs].hv[hh], i, SF::load(b.hv[hh], e));
}

}  // namespace

// ---------------------------------------------------------------- dispatch

#define QCD_SP_CASES(prec, SF, ...)                    \
    switch (prec) {                                    \
    case QCD_PREC_F64: {                               \
        using SF = SpF64;                              \
        __VA_ARGS__;                                   \
    } break;                                           \
    case QCD_PREC_F32: {                               \
        using SF = SpF32;                              \
        __VA_ARGS__;                                   \
    } break;                                           \
    case QCD_PREC_F16: {                               \
        using SF = SpF16;                              \
        __VA_ARGS__;                                   \
    } break;                                           \
    case QCD_PREC_BF16: {                              \
        using SF = SpBF16;                             \
        __VA_ARGS__;                                   \
    } break;                                           \
    case QCD_PREC_DF64: {                              \
        using SF = SpDF64;                             \
        __VA_ARGS__;                                   \
    } break;                                           \
    default:                                           \
        return cudaErrorInvalidValue;                  \
    }

static dim3 grid_of(const FieldView &f) { return dim3(site_blocks(nsites(f))); }

cudaError_t launch_convert(const FieldView &dst, const FieldView &src, cudaStream_t s)
{
    QCD_SP_CASES(dst.prec, SO, QCD_SP_CASES(src.prec, SI, convert_kernel<SO, SI><<<grid_of(dst), kThreads, 0, s>>>(dst, src)));
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_batch_copy(const FieldView &batched, const FieldView *plain, int n, int to_batch, cudaStream_t s)
{
    if (n < 1 || n > kMaxRhs || n > (1 << batched.rhs_log2)) return cudaErrorInvalidValue;
    PlainSet pl;
    for (int k = 0; k < n; ++k) {
        if (batched.prec != plain[k].prec || batched.nh != plain[k].nh || plain[k].h << batched.rhs_log2 != batched.h)
            return cudaErrorInvalidValue;
        pl.f[k] = plain[k];
    }
    QCD_SP_CASES(batched.prec, SF,
                 batch_copy_kernel<SF><<<grid_of(batched), kThreads, 0, s>>>(batched, pl, n, to_batch));
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_zero(const FieldView &f, cudaStream_t s)
{
    QCD_SP_CASES(f.prec, SF, zero_kernel<SF><<<grid_of(f), kThreads, 0, s>>>(f));
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_twist(const FieldView &out, const FieldView &in, const double c[2][2], cudaStream_t s,
                         const double *table, int stride)
{
    if (out.prec != in.prec) return cudaErrorInvalidValue;
    QCD_SP_CASES(out.prec, SF, twist_kernel<SF><<<grid_of(out), kThreads, 0, s>>>(out, in, c[0][0], c[0][1], c[1][0], c[1][1],
                                                                                 table, stride));
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_norm2(const FieldView &f, const Reduction &red, FinalizeKind fin, CgState *stt, double *out,
                         cudaStream_t s)
{
    if (!reduction_fits(red, 1, f.rhs_log2, grid_of(f).x)) return cudaErrorInvalidValue;
    QCD_SP_CASES(f.prec, SF, norm2_kernel<SF><<<grid_of(f), kThreads, 0, s>>>(f, red, fin, stt, out));
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_diff_norm2(const FieldView &a, const FieldView &b, const Reduction &red, double *out, cudaStream_t s)
{
    if (a.prec != QCD_PREC_F64 || b.prec != QCD_PREC_F64) return cudaErrorInvalidValue;
    if (!reduction_fits(red, 2, a.rhs_log2, grid_of(a).x)) return cudaErrorInvalidValue;
    diff_norm2_kernel<<<grid_of(a), kThreads, 0, s>>>(a, b, red, out);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_cg_state_init(CgState *stt, int nrhs, const RhsValues &tol2, double delta2, int maxiter,
                                 cudaStream_t s)
{
    cg_state_init_kernel<<<1, 1, 0, s>>>(stt, nrhs, tol2, delta2, maxiter);
    note_launches();
    return cudaGetLastError();
}


cudaError_t launch_cg_ctrl_reliable(const CgState *stt, cudaGraphConditionalHandle h, cudaStream_t s)
{
    cg_ctrl_reliable_kernel<<<1, 1, 0, s>>>(stt, h);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_cg_ctrl_loop(CgState *stt, cudaGraphConditionalHandle h, cudaStream_t s)
{
    cg_ctrl_loop_kernel<<<1, 1, 0, s>>>(stt, h);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_cg_setup(const FieldView &rhs, const FieldView &r, const FieldView &p, const FieldView &x,
                            const FieldView *xs, const Reduction &red, CgState *stt, cudaStream_t s)
{
    const FieldView xsv = xs ? *xs : x;
    const bool has = xs != nullptr;
    if (!reduction_fits(red, 1, rhs.rhs_log2, grid_of(rhs).x)) return cudaErrorInvalidValue;
    if (x.prec == QCD_PREC_F64 && r.prec == QCD_PREC_F64 && !has) {
        cg_setup_kernel<SpF64, SpF64, SpF32><<<grid_of(rhs), kThreads, 0, s>>>(rhs, r, p, x, xsv, false, red, stt);
    } else if (x.prec == QCD_PREC_F64 && has && xs->prec == QCD_PREC_DF64 && r.prec == QCD_PREC_DF64) {
        cg_setup_kernel<SpDF64, SpF64, SpDF64><<<grid_of(rhs), kThreads, 0, s>>>(rhs, r, p, x, xsv, true, red, stt);
    } else if (x.prec == QCD_PREC_F64 && has && xs->prec == QCD_PREC_F32) {
        QCD_SP_CASES(r.prec, SR,
                     cg_setup_kernel<SR, SpF64, SpF32><<<grid_of(rhs), kThreads, 0, s>>>(rhs, r, p, x, xsv, true, red, stt));
    } else {
        return cudaErrorInvalidValue;
    }
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_cg_xr(const FieldView &x, const FieldView &p, const FieldView &r, const FieldView &q,
                         const Reduction &red, CgState *stt, cudaStream_t s)
{
    if (!reduction_fits(red, 1, x.rhs_log2, grid_of(x).x)) return cudaErrorInvalidValue;
    if (x.prec == QCD_PREC_F64 && p.prec == QCD_PREC_F64) {
        cg_xr_kernel<SpF64, SpF64><<<grid_of(x), kThreads, 0, s>>>(x, p, r, q, red, stt);
    } else if (x.prec == QCD_PREC_DF64 && p.prec == QCD_PREC_DF64) {
        cg_xr_kernel<SpDF64, SpDF64><<<grid_of(x), kThreads, 0, s>>>(x, p, r, q, red, stt);
    } else if (x.prec == QCD_PREC_F32) {
        QCD_SP_CASES(p.prec, SF, cg_xr_kernel<SpF32, SF><<<grid_of(x), kThreads, 0, s>>>(x, p, r, q, red, stt));
    } else {
        return cudaErrorInvalidValue;
    }
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_cg_p(const FieldView &p, const FieldView &r, CgState *stt, cudaStream_t s)
{
    QCD_SP_CASES(p.prec, SF, cg_p_kernel<SF><<<grid_of(p), kThreads, 0, s>>>(p, r, stt));
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_cg_accum_x(const FieldView &xhi, const FieldView &xs, cudaStream_t s)
{
    QCD_SP_CASES(xs.prec, SS, cg_accum_x_kernel<SS><<<grid_of(xhi), kThreads, 0, s>>>(xhi, xs));
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_cg_defect(const FieldView &rhs0, const FieldView &q, const FieldView &rho, const FieldView &rs,
                             cudaStream_t s)
{
    QCD_SP_CASES(rs.prec, SS, cg_defect_kernel<SS><<<grid_of(rhs0), kThreads, 0, s>>>(rhs0, q, rho, rs));
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_cg_verify(const FieldView &f, const Reduction &red, CgState *stt, cudaStream_t s)
{
    if (!reduction_fits(red, 1, f.rhs_log2, grid_of(f).x)) return cudaErrorInvalidValue;
    cg_verify_kernel<<<grid_of(f), kThreads, 0, s>>>(f, red, stt);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_cg_true_residual(const FieldView &rhs, const FieldView &q, const FieldView &rhi, const FieldView *rs,
                                    const Reduction &red, CgState *stt, cudaStream_t s)
{
    if (!reduction_fits(red, 1, rhs.rhs_log2, grid_of(rhs).x)) return cudaErrorInvalidValue;
    if (!rs) {
        cg_true_residual_kernel<SpF64><<<grid_of(rhs), kThreads, 0, s>>>(rhs, q, rhi, rhi, false, red, stt);
    } else {
        QCD_SP_CASES(rs->prec, SS,
                     cg_true_residual_kernel<SS><<<grid_of(rhs), kThreads, 0, s>>>(rhs, q, rhi, *rs, true, red, stt));
    }
    note_launches();
    return cudaGetLastError();
}

}  // namespace qcd
