// Even-odd Wilson hopping kernel D_eo / D_oe (and their adjoints) with a
// fused epilogue, templated on the storage formats.
//
// The operation is the "Dslash" of CL2QCD (arXiv:1411.5219, Sec. 1): the
// derivative part of the Wilson matrix, applied many times per inversion
// and limited by memory bandwidth.  For an output site x of parity p:
//
//   (D psi)(x) = sum_mu (1 - S gamma_mu) U_mu(x) psi(x+mu)
//                     + (1 + S gamma_mu) U_mu(x-mu)^dagger psi(x-mu),
//
// S = +1 for D and S = -1 for D^dagger (the adjoint swaps the projectors),
// psi lives on the sites of parity 1-p.  Each neighbour spinor is projected
// to a two-spin half spinor h = psi_up - S B psi_dn (gamma_mu = [[0, B],
// [B^dagger, 0]] in the chiral basis), the link multiplies the two colour
// vectors of h, and the lower spins are rebuilt as -S B^dagger (U h).
//
// One thread computes one output site.  Links of the forward hops are read
// at the output site (block (p, mu)), links of the backward hops at the
// neighbour (block (1-p, mu)), so every link is read exactly once per call.
#pragma once

#include "qcd_internal.cuh"

namespace qcd {

template <typename R, int MU, int S>
__device__ __forceinline__ HalfSpinor<R> project(const Spinor<R> &p)
{
    HalfSpinor<R> h;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (MU == 0) {  // B = -i sigma_1: h = (psi0 + S i psi3, psi1 + S i psi2)
            h.c[0][c] = S > 0 ? p.c[0][c] + ti(p.c[3][c]) : p.c[0][c] - ti(p.c[3][c]);
            h.c[1][c] = S > 0 ? p.c[1][c] + ti(p.c[2][c]) : p.c[1][c] - ti(p.c[2][c]);
        } else if (MU == 1) {  // B = -i sigma_2: h = (psi0 + S psi3, psi1 - S psi2)
            h.c[0][c] = S > 0 ? p.c[0][c] + p.c[3][c] : p.c[0][c] - p.c[3][c];
            h.c[1][c] = S > 0 ? p.c[1][c] - p.c[2][c] : p.c[1][c] + p.c[2][c];
        } else if (MU == 2) {  // B = -i sigma_3: h = (psi0 + S i psi2, psi1 - S i psi3)
            h.c[0][c] = S > 0 ? p.c[0][c] + ti(p.c[2][c]) : p.c[0][c] - ti(p.c[2][c]);
            h.c[1][c] = S > 0 ? p.c[1][c] - ti(p.c[3][c]) : p.c[1][c] + ti(p.c[3][c]);
        } else {  // B = 1: h = (psi0 - S psi2, psi1 - S psi3)
            h.c[0][c] = S > 0 ? p.c[0][c] - p.c[2][c] : p.c[0][c] + p.c[2][c];
            h.c[1][c] = S > 0 ? p.c[1][c] - p.c[3][c] : p.c[1][c] + p.c[3][c];
        }
    }
    return h;
}

// acc (+)= the full spinor rebuilt from the multiplied half spinor u:
// upper = u, lower = -S B^dagger u.
template <typename R, int MU, int S, bool kFirst>
__device__ __forceinline__ void accumulate(Spinor<R> &acc, const HalfSpinor<R> &u)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cx<R> l2, l3;
        if (MU == 0) {  // -S (i u1, i u0)
            l2 = S > 0 ? -ti(u.c[1][c]) : ti(u.c[1][c]);
            l3 = S > 0 ? -ti(u.c[0][c]) : ti(u.c[0][c]);
        } else if (MU == 1) {  // -S (u1, -u0)
            l2 = S > 0 ? -u.c[1][c] : u.c[1][c];
            l3 = S > 0 ? u.c[0][c] : -u.c[0][c];
        } else if (MU == 2) {  // -S (i u0, -i u1)
            l2 = S > 0 ? -ti(u.c[0][c]) : ti(u.c[0][c]);
            l3 = S > 0 ? ti(u.c[1][c]) : -ti(u.c[1][c]);
        } else {  // -S (u0, u1)
            l2 = S > 0 ? -u.c[0][c] : u.c[0][c];
            l3 = S > 0 ? -u.c[1][c] : u.c[1][c];
        }
        if (kFirst) {
            acc.c[0][c] = u.c[0][c];
            acc.c[1][c] = u.c[1][c];
            acc.c[2][c] = l2;
            acc.c[3][c] = l3;
        } else {
            acc.c[0][c] = acc.c[0][c] + u.c[0][c];
            acc.c[1][c] = acc.c[1][c] + u.c[1][c];
            acc.c[2][c] = acc.c[2][c] + l2;
            acc.c[3][c] = acc.c[3][c] + l3;
        }
    }
}

// U h (kAdj = false) or U^dagger h (kAdj = true) on both colour vectors.
template <typename R, bool kAdj>
__device__ __forceinline__ HalfSpinor<R> su3_mul(const Link<R> &u, const HalfSpinor<R> &h)
{
    HalfSpinor<R> r;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!kAdj) {
                cx<R> v = cmul(u.m[a][0], h.c[s][0]);
                v = cmac(v, u.m[a][1], h.c[s][1]);
                v = cmac(v, u.m[a][2], h.c[s][2]);
                r.c[s][a] = v;
            } else {
                cx<R> v = cjmul(u.m[0][a], h.c[s][0]);
                v = cjmac(v, u.m[1][a], h.c[s][1]);
                v = cjmac(v, u.m[2][a], h.c[s][2]);
                r.c[s][a] = v;
            }
        }
    return r;
}

template <typename R>
__device__ __forceinline__ void negate(HalfSpinor<R> &h)
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) h.c[s][c] = -h.c[s][c];
}

// One hop: load the neighbour spinor and the link, project, multiply,
// rebuild and accumulate.  `flip` applies the boundary factor -1.
template <typename SF, typename GF, int MU, int S, bool kAdj, bool kFirst>
__device__ __forceinline__ void hop(Spinor<typename SF::R> &acc, const SpinorView &in, const GaugeView &U, int nb,
                                    int lblock, int lidx, bool flip)
{
    using R = typename SF::R;
    const Spinor<R> psi = SF::load(in, nb);
    const Link<R> u = GF::load(U, lblock, lidx);
    HalfSpinor<R> h = project<R, MU, S>(psi);
    HalfSpinor<R> uh = su3_mul<R, kAdj>(u, h);
    if (flip) negate(uh);
    accumulate<R, MU, S, kFirst>(acc, uh);
}

template <typename SF, typename GF, int kDagger, int kEpi, bool kReduce>
__global__ void __launch_bounds__(kThreads) dslash_kernel(const DslashLaunch a)
{
    using R = typename SF::R;
    if (a.check_status && a.state->status != CG_RUNNING) return;
    constexpr int SF_ = kDagger ? -1 : +1;  // projector sign of forward hops
    constexpr int SB_ = -SF_;                // ... of backward hops
    const int nbp = (a.g.h + kThreads - 1) / kThreads;
    const int p = a.both ? (int)(blockIdx.x >= (unsigned)nbp) : a.out_parity;
    const int i = (blockIdx.x - (a.both ? p * nbp : 0)) * blockDim.x + threadIdx.x;
    double red[1] = {0.0};
    if (i < a.g.h) {
        const Geom &g = a.g;
        const SpinorView &in = a.in[p];
        const SiteCoords c = site_coords(g, i, p);
        const int base = i - c.xh;
        const int fwd = p * 4, bwd = (1 - p) * 4;
        Spinor<R> acc;
        // x
        {
            const int xf = c.x + 1 == g.L[0] ? 0 : c.x + 1;
            const int xb = c.x == 0 ? g.L[0] - 1 : c.x - 1;
            const int nf = base + (xf >> 1), nbk = base + (xb >> 1);
            hop<SF, GF, 0, SF_, false, true>(acc, in, a.U, nf, fwd + 0, i, false);
            hop<SF, GF, 0, SB_, true, false>(acc, in, a.U, nbk, bwd + 0, nbk, false);
        }
        // y
        {
            const int nf = c.y == g.L[1] - 1 ? i - (g.L[1] - 1) * g.sy : i + g.sy;
            const int nbk = c.y == 0 ? i + (g.L[1] - 1) * g.sy : i - g.sy;
            hop<SF, GF, 1, SF_, false, false>(acc, in, a.U, nf, fwd + 1, i, false);
            hop<SF, GF, 1, SB_, true, false>(acc, in, a.U, nbk, bwd + 1, nbk, false);
        }
        // z
        {
            const int nf = c.z == g.L[2] - 1 ? i - (g.L[2] - 1) * g.sz : i + g.sz;
            const int nbk = c.z == 0 ? i + (g.L[2] - 1) * g.sz : i - g.sz;
            hop<SF, GF, 2, SF_, false, false>(acc, in, a.U, nf, fwd + 2, i, false);
            hop<SF, GF, 2, SB_, true, false>(acc, in, a.U, nbk, bwd + 2, nbk, false);
        }
        // t (boundary factor on the wrapping hop)
        {
            const bool wf = c.t == g.L[3] - 1, wb = c.t == 0;
            const int nf = wf ? i - (g.L[3] - 1) * g.st : i + g.st;
            const int nbk = wb ? i + (g.L[3] - 1) * g.st : i - g.st;
            const bool anti = g.tbc < 0.0;
            hop<SF, GF, 3, SF_, false, false>(acc, in, a.U, nf, fwd + 3, i, anti && wf);
            hop<SF, GF, 3, SB_, true, false>(acc, in, a.U, nbk, bwd + 3, nbk, anti && wb);
        }
        // epilogue
        Spinor<R> out;
        if (kEpi == EPI_PLAIN) {
            out = acc;
        } else if (kEpi == EPI_REAL_D) {
            const R d = (R)a.cd[0][0];
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) out.c[s][cc] = d * acc.c[s][cc];
        } else if (kEpi == EPI_REAL_YD) {
            const Spinor<R> y = SF::load(a.y[p], i);
            const R cy = (R)a.cy[0][0], d = (R)a.cd[0][0];
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    out.c[s][cc].re = fma(d, acc.c[s][cc].re, cy * y.c[s][cc].re);
                    out.c[s][cc].im = fma(d, acc.c[s][cc].im, cy * y.c[s][cc].im);
                }
        } else {
            const cx<R> d[2] = {mk((R)a.cd[0][0], (R)a.cd[0][1]), mk((R)a.cd[1][0], (R)a.cd[1][1])};
            if (kEpi == EPI_CPLX_D) {
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) out.c[s][cc] = cmul(d[s >> 1], acc.c[s][cc]);
            } else {
                const Spinor<R> y = SF::load(a.y[p], i);
                const cx<R> cy[2] = {mk((R)a.cy[0][0], (R)a.cy[0][1]), mk((R)a.cy[1][0], (R)a.cy[1][1])};
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) out.c[s][cc] = cmac(cmul(cy[s >> 1], y.c[s][cc]), d[s >> 1], acc.c[s][cc]);
            }
        }
        SF::store(a.out[p], i, out);
        if (kReduce) {
            R n = 0;
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) n += out.c[s][cc].re * out.c[s][cc].re + out.c[s][cc].im * out.c[s][cc].im;
            red[0] = (double)n;
        }
    }
    if (kReduce) grid_reduce<1>(red, a.red, a.fin, a.state, a.red_out);
}

// Dispatch over dagger / epilogue / reduction for one format pair.
template <typename SF, typename GF>
cudaError_t launch_dslash_fmt(const DslashLaunch &a, cudaStream_t s)
{
    const dim3 grid(site_blocks(a.g.h) * (a.both ? 2 : 1)), block(kThreads);
#define QCD_DSL(D, E, RD)                                                   \
    if (a.dagger == D && a.epi == E && a.reduce == RD) {                    \
        dslash_kernel<SF, GF, D, E, RD><<<grid, block, 0, s>>>(a);          \
        return cudaGetLastError();                                          \
    }
#define QCD_DSL_E(D, E) QCD_DSL(D, E, false) QCD_DSL(D, E, true)
#define QCD_DSL_D(D)                                                        \
    QCD_DSL(D, EPI_PLAIN, false)                                            \
    QCD_DSL(D, EPI_REAL_D, false)                                           \
    QCD_DSL(D, EPI_CPLX_D, false)                                           \
    QCD_DSL_E(D, EPI_REAL_YD) QCD_DSL_E(D, EPI_CPLX_YD)
    QCD_DSL_D(0)
    QCD_DSL_D(1)
#undef QCD_DSL_D
#undef QCD_DSL_E
#undef QCD_DSL
    return cudaErrorInvalidValue;
}

}  // namespace qcd
