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
#include "dslash_pairs.cuh"
#include "hop_lanes.cuh"

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
template <typename R>
__device__ __forceinline__ cx<R> wadd(cx<R> acc, R w, cx<R> v)
{
    return {fma(w, v.re, acc.re), fma(w, v.im, acc.im)};
}

// kW: the hop carries a weight w (the FP16 per-site scale, with the
// boundary sign), applied in the accumulating FMAs.
template <typename R, int MU, int S, bool kFirst, bool kW>
__device__ __forceinline__ void accumulate(Spinor<R> &acc, const HalfSpinor<R> &u, R w)
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
        if (kFirst && kW) {
            acc.c[0][c] = w * u.c[0][c];
            acc.c[1][c] = w * u.c[1][c];
            acc.c[2][c] = w * l2;
            acc.c[3][c] = w * l3;
        } else if (kFirst) {
            acc.c[0][c] = u.c[0][c];
            acc.c[1][c] = u.c[1][c];
            acc.c[2][c] = l2;
            acc.c[3][c] = l3;
        } else if (kW) {
            acc.c[0][c] = wadd(acc.c[0][c], w, u.c[0][c]);
            acc.c[1][c] = wadd(acc.c[1][c], w, u.c[1][c]);
            acc.c[2][c] = wadd(acc.c[2][c], w, l2);
            acc.c[3][c] = wadd(acc.c[3][c], w, l3);
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

// seed + U h (kAdj = false) or seed + U^dagger h (kAdj = true): the
// product's multiply-add chains start from the seed.
template <typename R, bool kAdj>
__device__ __forceinline__ HalfSpinor<R> su3_mul_seeded(const Link<R> &u, const HalfSpinor<R> &h,
                                                        const HalfSpinor<R> &seed)
{
    HalfSpinor<R> r;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<R> v = seed.c[s][a];
#pragma unroll
            for (int j = 0; j < 3; ++j) v = kAdj ? cjmac(v, u.m[j][a], h.c[s][j]) : cmac(v, u.m[a][j], h.c[s][j]);
            r.c[s][a] = v;
        }
    return r;
}

// Both hops of direction mu at once (FP64 kernels): with u_f = U h_f of
// the forward hop and u_b = U^dagger h_b of the backward one, the upper spins
// gain s = u_f + u_b and the lower spins phi pi(u_f - u_b), since the two
// hops' rebuild phases differ only in sign.  s comes from the backward
// product's chains seeded with u_f, and u_f - u_b = 2 u_f - s, which saves
// the separate additions of one hop.
template <typename R, int MU, int S, bool kFirst>
__device__ __forceinline__ void accumulate_pair(Spinor<R> &acc, const HalfSpinor<R> &uf, const HalfSpinor<R> &sum)
{
    HalfSpinor<R> d;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            d.c[s][c].re = fma(R(2), uf.c[s][c].re, -sum.c[s][c].re);
            d.c[s][c].im = fma(R(2), uf.c[s][c].im, -sum.c[s][c].im);
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cx<R> l2, l3;
        if (MU == 0) {  // -S (i d1, i d0)
            l2 = S > 0 ? -ti(d.c[1][c]) : ti(d.c[1][c]);
            l3 = S > 0 ? -ti(d.c[0][c]) : ti(d.c[0][c]);
        } else if (MU == 1) {  // -S (d1, -d0)
            l2 = S > 0 ? -d.c[1][c] : d.c[1][c];
            l3 = S > 0 ? d.c[0][c] : -d.c[0][c];
        } else if (MU == 2) {  // -S (i d0, -i d1)
            l2 = S > 0 ? -ti(d.c[0][c]) : ti(d.c[0][c]);
            l3 = S > 0 ? ti(d.c[1][c]) : -ti(d.c[1][c]);
        } else {  // -S (d0, d1)
            l2 = S > 0 ? -d.c[0][c] : d.c[0][c];
            l3 = S > 0 ? -d.c[1][c] : d.c[1][c];
        }
        if (kFirst) {
            acc.c[0][c] = sum.c[0][c];
            acc.c[1][c] = sum.c[1][c];
            acc.c[2][c] = l2;
            acc.c[3][c] = l3;
        } else {
            acc.c[0][c] = acc.c[0][c] + sum.c[0][c];
            acc.c[1][c] = acc.c[1][c] + sum.c[1][c];
            acc.c[2][c] = acc.c[2][c] + l2;
            acc.c[3][c] = acc.c[3][c] + l3;
        }
    }
}

template <typename R>
__device__ __forceinline__ void negate(HalfSpinor<R> &h)
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) h.c[s][c] = -h.c[s][c];
}

// The forward hop of a pair: u_f = U h_f (flip: h_f negated).
template <typename SF, typename GF, int MU, int S>
__device__ __forceinline__ HalfSpinor<typename SF::R> hop_fwd(const typename SF::Raw &rs, const typename GF::Raw &ru,
                                                               bool flip)
{
    using R = typename SF::R;
    HalfSpinor<R> h = project<R, MU, S>(SF::decode(rs));
    if (flip) negate(h);
    return su3_mul<R, false>(GF::decode(ru), h);
}

// The backward hop of a pair, accumulated with the forward result uf.
template <typename SF, typename GF, int MU, int SFW, int SBW, bool kFirst>
__device__ __forceinline__ void hop_bwd(Spinor<typename SF::R> &acc, const HalfSpinor<typename SF::R> &uf,
                                        const typename SF::Raw &rs, const typename GF::Raw &ru, bool flip)
{
    using R = typename SF::R;
    HalfSpinor<R> h = project<R, MU, SBW>(SF::decode(rs));
    if (flip) negate(h);
    const HalfSpinor<R> sum = su3_mul_seeded<R, true>(GF::decode(ru), h, uf);
    accumulate_pair<R, MU, SFW, kFirst>(acc, uf, sum);
}

// One hop from already fetched raw data: decode, project, multiply,
// rebuild and accumulate.  `flip` applies the boundary factor -1.
template <typename SF, typename GF, int MU, int S, bool kAdj, bool kFirst>
__device__ __forceinline__ void hop(Spinor<typename SF::R> &acc, const typename SF::Raw &rs,
                                    const typename GF::Raw &ru, bool flip)
{
    using R = typename SF::R;
    const Spinor<R> psi = SF::decode(rs);
    const Link<R> u = GF::decode(ru);
    const HalfSpinor<R> h = project<R, MU, S>(psi);
    HalfSpinor<R> uh = su3_mul<R, kAdj>(u, h);
    if (SF::kScaled) {
        const R w = flip ? -SF::scale(rs) : SF::scale(rs);
        accumulate<R, MU, S, kFirst, true>(acc, uh, w);
    } else {
        if (flip) negate(uh);
        accumulate<R, MU, S, kFirst, false>(acc, uh, R(1));
    }
}

// Threads per block: FP64 kernels hold ~170 registers (2-3 blocks of 128
// per SM), so they use blocks of 64 to spread the grid evenly over the 152
// SMs; the FP32/16-bit kernels use 128.
template <typename SF>
__host__ __device__ constexpr int dslash_tpb()
{
    return sizeof(typename SF::R) == 8 ? 64 : 128;
}

// Blocks per SM the register budget must allow: six 64-thread FP64 blocks
// (<= 170 registers) put a 24^3 x 8 half lattice (864 blocks) in a single
// wave on 152 SMs.
template <typename SF>
__host__ __device__ constexpr int dslash_min_blocks()
{
    return sizeof(typename SF::R) == 8 ? 6 : 1;
}

// Minimum resident blocks for __launch_bounds__: the FP64-family kernels at
// 64 threads need six (<= 170 registers); the 16-bit kernels with 16-bit
// links (mixed-precision products, 120-122 registers uncapped) five blocks of 128
// or ten of 64 (96 registers, 20 warps per SM instead of 16, to hide their
// memory latency); the other 4-byte kernels are not capped (64- and
// 85-register caps spill and measured slower at 24^3x8 and 48^3x12), nor is
// FP64 reconstruct-8, whose rebuild would spill under the cap.
template <typename SF, typename GF, int TPB>
__host__ __device__ constexpr int dslash_min_blocks_tpb()
{
    if constexpr (sizeof(typename SF::R) == 8 && GF::kRecon_ != 8) return TPB == 64 ? 6 : 1;
    if constexpr (is_mixed16<SF, GF>::value) return TPB == 64 ? 10 : TPB == 128 ? 5 : 2;
    return 1;
}

template <typename SF, typename GF, int kDagger, int kEpi, bool kReduce, int TPB,
          int kMinBlocks = dslash_min_blocks_tpb<SF, GF, TPB>()>
__global__ void __launch_bounds__(TPB, kMinBlocks) dslash_kernel(const DslashLaunch a)
{
    using R = typename SF::R;
    if (a.check_status && a.state->status != a.run_status) return;
    constexpr int SF_ = kDagger ? -1 : +1;  // projector sign of forward hops
    constexpr int SB_ = -SF_;                // ... of backward hops
    // element e = site i * 2^rhs_log2 + rhs (one rhs: e = i)
    const int ne = a.g.h << a.rhs_log2;
    const int nbp = (ne + TPB - 1) / TPB;
    const int p = a.both ? (int)(blockIdx.x >= (unsigned)nbp) : a.out_parity;
    int bl = blockIdx.x - (a.both ? p * nbp : 0);
    // with tmap = blocks per time slice, consecutive blocks take the same
    // space chunk at consecutive t, so every neighbour is re-read within a
    // few MB of traffic (an L2 hit) even when a batched field exceeds L2
    if (a.tmap) bl = (bl % a.g.L[3]) * a.tmap + bl / a.g.L[3];
    const int e = bl * blockDim.x + threadIdx.x;
    const int L = a.rhs_log2, rhs = e & ((1 << L) - 1);
    const int i = e >> L;
    // fused norm: summed within the warp in float by the FP32/16-bit kernels
    using RedT = typename std::conditional<std::is_same<R, float>::value, float, double>::type;
    RedT red[1] = {RedT(0)};
    if (e < ne) {
        const Geom &g = a.g;
        const SpinorView &in = a.in[p];
        const SiteCoords c = site_coords(g, i, p);
        const int base = i - c.xh;
        const int fwd = p * 4, bwd = (1 - p) * 4;
        // neighbour half-site, link block and link index of the 8 hops in
        // the order x+, x-, y+, y-, z+, z-, t+, t-
        int nb[8], lb[8], li[8];
        bool fl[8];
        {
            const int xf = c.x + 1 == g.L[0] ? 0 : c.x + 1;
            const int xb = c.x == 0 ? g.L[0] - 1 : c.x - 1;
            nb[0] = base + (xf >> 1);
            nb[1] = base + (xb >> 1);
            nb[2] = c.y == g.L[1] - 1 ? i - (g.L[1] - 1) * g.sy : i + g.sy;
            nb[3] = c.y == 0 ? i + (g.L[1] - 1) * g.sy : i - g.sy;
            nb[4] = c.z == g.L[2] - 1 ? i - (g.L[2] - 1) * g.sz : i + g.sz;
            nb[5] = c.z == 0 ? i + (g.L[2] - 1) * g.sz : i - g.sz;
            const bool wf = c.t == g.L[3] - 1, wb = c.t == 0;
            nb[6] = wf ? i - (g.L[3] - 1) * g.st : i + g.st;
            nb[7] = wb ? i + (g.L[3] - 1) * g.st : i - g.st;
            const bool anti = antiperiodic(g);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                lb[k] = (k & 1 ? bwd : fwd) + (k >> 1);
                li[k] = k & 1 ? nb[k] : i;
                nb[k] = (nb[k] << L) | rhs;  // neighbour element of the same rhs
                fl[k] = false;
            }
            fl[6] = anti && wf;
            fl[7] = anti && wb;
        }
        Spinor<R> acc;
        // software pipeline: the loads of hop k+1 are issued before the
        // arithmetic of hop k
        typename SF::Raw rs = SF::fetch(in, nb[0]);
        typename GF::Raw ru = GF::fetch(a.U, lb[0], li[0]);
#define QCD_HOP(K, MU, S, ADJ, FIRST)                                        \
    {                                                                      \
        typename SF::Raw rs_n;                                             \
        typename GF::Raw ru_n;                                             \
        if (K < 7) {                                                       \
            rs_n = SF::fetch(in, nb[(K + 1) & 7]);                         \
            ru_n = GF::fetch(a.U, lb[(K + 1) & 7], li[(K + 1) & 7]);       \
        }                                                                  \
        hop<SF, GF, MU, S, ADJ, FIRST>(acc, rs, ru, fl[K]);                \
        if (K < 7) {                                                       \
            rs = rs_n;                                                     \
            ru = ru_n;                                                     \
        }                                                                  \
    }
        if constexpr (uses_pairs<SF>::value) {
            // 16-bit and FP32 spinors: packed FP32 arithmetic on the two spins
            AccPairs ap;
#define QCD_HOP16(K, MU, S, ADJ, FIRST)                                      \
    {                                                                      \
        typename SF::Raw rs_n;                                             \
        typename GF::Raw ru_n;                                             \
        if (K < 7) {                                                       \
            rs_n = SF::fetch(in, nb[(K + 1) & 7]);                         \
            ru_n = GF::fetch(a.U, lb[(K + 1) & 7], li[(K + 1) & 7]);       \
        }                                                                  \
        hop_pairs<SF, GF, MU, S, ADJ, FIRST>(ap, rs, ru, fl[K]);           \
        if (K < 7) {                                                       \
            rs = rs_n;                                                     \
            ru = ru_n;                                                     \
        }                                                                  \
    }
            QCD_HOP16(0, 0, SF_, false, true)
            QCD_HOP16(1, 0, SB_, true, false)
            QCD_HOP16(2, 1, SF_, false, false)
            QCD_HOP16(3, 1, SB_, true, false)
            QCD_HOP16(4, 2, SF_, false, false)
            QCD_HOP16(5, 2, SB_, true, false)
            QCD_HOP16(6, 3, SF_, false, false)
            QCD_HOP16(7, 3, SB_, true, false)
#undef QCD_HOP16
            acc = unpair(ap);
        } else if constexpr (!std::is_same<R, double>::value) {
            QCD_HOP(0, 0, SF_, false, true)
            QCD_HOP(1, 0, SB_, true, false)
            QCD_HOP(2, 1, SF_, false, false)
            QCD_HOP(3, 1, SB_, true, false)
            QCD_HOP(4, 2, SF_, false, false)
            QCD_HOP(5, 2, SB_, true, false)
            QCD_HOP(6, 3, SF_, false, false)
            QCD_HOP(7, 3, SB_, true, false)
        } else {
            // FP64 (bound by FP64 instructions): the two hops of each
            // direction as a pair, 48 fewer FP64 instructions per site
            // (measured 5 % faster at 48^3x12); the 4-byte kernels would need
            // ~230 registers for it
            HalfSpinor<R> uf;
#define QCD_PAIR(K, MU, FIRST)                                                         \
    {                                                                                  \
        typename SF::Raw rs_n = SF::fetch(in, nb[K + 1]);                              \
        typename GF::Raw ru_n = GF::fetch(a.U, lb[K + 1], li[K + 1]);                  \
        uf = hop_fwd<SF, GF, MU, SF_>(rs, ru, fl[K]);                                  \
        rs = rs_n;                                                                     \
        ru = ru_n;                                                                     \
        if (K + 1 < 7) {                                                               \
            rs_n = SF::fetch(in, nb[(K + 2) & 7]);                                     \
            ru_n = GF::fetch(a.U, lb[(K + 2) & 7], li[(K + 2) & 7]);                   \
        }                                                                              \
        hop_bwd<SF, GF, MU, SF_, SB_, FIRST>(acc, uf, rs, ru, fl[K + 1]);              \
        if (K + 1 < 7) {                                                               \
            rs = rs_n;                                                                 \
            ru = ru_n;                                                                 \
        }                                                                              \
    }
            QCD_PAIR(0, 0, true)
            QCD_PAIR(2, 1, false)
            QCD_PAIR(4, 2, false)
            QCD_PAIR(6, 3, false)
#undef QCD_PAIR
        }
#undef QCD_HOP
        // epilogue coefficients: kernel parameters, or a device table shared
        // by every launch of a captured CG graph (so one graph serves all
        // kappa and mu)
        // (with a per-rhs table, the one of this element's rhs).  The FP32 and
        // 16-bit kernels read float copies: a double-to-float conversion would
        // occupy the FP64 pipe once per coefficient and thread.  The source is
        // chosen by a branch on the kernel parameter: a per-thread select
        // between a table load and a parameter cost the FP32 epilogue
        // variants ~70 registers (226 instead of 155).
        constexpr bool kF32 = std::is_same<R, float>::value;
        using CR = typename std::conditional<kF32, float, double>::type;
        CR cyv[2][2], cdv[2][2];
        if constexpr (kF32) {
            if (a.coef_f) {
                const float *cf = a.coef_f + (size_t)rhs * a.coef_stride;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    cyv[k >> 1][k & 1] = __ldg(cf + k);
                    cdv[k >> 1][k & 1] = __ldg(cf + 4 + k);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    cyv[k >> 1][k & 1] = a.cyf[k >> 1][k & 1];
                    cdv[k >> 1][k & 1] = a.cdf[k >> 1][k & 1];
                }
            }
        } else {
            if (a.coef) {
                const double *cf = a.coef + (size_t)rhs * a.coef_stride;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    cyv[k >> 1][k & 1] = __ldg(cf + k);
                    cdv[k >> 1][k & 1] = __ldg(cf + 4 + k);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    cyv[k >> 1][k & 1] = a.cy[k >> 1][k & 1];
                    cdv[k >> 1][k & 1] = a.cd[k >> 1][k & 1];
                }
            }
        }
        // epilogue
        Spinor<R> out;
        if (kEpi == EPI_PLAIN) {
            out = acc;
        } else if (kEpi == EPI_REAL_D) {
            const R d = (R)cdv[0][0];
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) out.c[s][cc] = d * acc.c[s][cc];
        } else if (kEpi == EPI_REAL_YD) {
            const Spinor<R> y = SF::load(a.y[p], e);
            const R cy = (R)cyv[0][0], d = (R)cdv[0][0];
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    out.c[s][cc].re = fma(d, acc.c[s][cc].re, cy * y.c[s][cc].re);
                    out.c[s][cc].im = fma(d, acc.c[s][cc].im, cy * y.c[s][cc].im);
                }
        } else {
            const cx<R> d[2] = {mk((R)cdv[0][0], (R)cdv[0][1]), mk((R)cdv[1][0], (R)cdv[1][1])};
            if (kEpi == EPI_CPLX_D) {
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) out.c[s][cc] = cmul(d[s >> 1], acc.c[s][cc]);
            } else {
                const Spinor<R> y = SF::load(a.y[p], e);
                const cx<R> cy[2] = {mk((R)cyv[0][0], (R)cyv[0][1]), mk((R)cyv[1][0], (R)cyv[1][1])};
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) out.c[s][cc] = cmac(cmul(cy[s >> 1], y.c[s][cc]), d[s >> 1], acc.c[s][cc]);
            }
        }
        SF::store(a.out[p], e, out);
        if (kReduce) {
            R n = 0;
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) n += out.c[s][cc].re * out.c[s][cc].re + out.c[s][cc].im * out.c[s][cc].im;
            red[0] = (RedT)n;
        }
    }
    if (kReduce) grid_reduce_rhs<1>(red, a.rhs_log2, a.red, a.fin, a.state, a.red_out);
}

// Dispatch over epilogue / reduction for one format pair, one dagger value
// and one block size.  (The real-scale epilogue without y has no caller and
// is not instantiated.)
// FP64 reconstruct-18, one right-hand side: eight threads per site, one hop
// each (hop_lanes.cuh), for small lattices whose time a single thread's
// chain of FP64 hops would set.  Same epilogues and fused reduction as
// dslash_kernel; lanes with bit 0 clear own one spin of the output.
template <int kDagger, int kEpi, bool kReduce>
__global__ void __launch_bounds__(128) dslash_lanes8_kernel(const DslashLaunch a)
{
    if (a.check_status && a.state->status != a.run_status) return;
    const int items = a.g.h * 8;
    const int nbp = (items + 127) / 128;
    const int p = a.both ? (int)(blockIdx.x >= (unsigned)nbp) : a.out_parity;
    const int w = (blockIdx.x - (a.both ? p * nbp : 0)) * 128 + threadIdx.x;
    const bool act = w < items;
    const int i = w >> 3, lane = w & 7;
    cx<double> acc[12];
    if (act) {
        hop_lane8<false>(a.g, static_cast<const double2 *>(a.U.data), a.U.stride,
                         static_cast<const double2 *>(a.in[p].data), a.in[p].stride, p, i, lane, kDagger != 0, acc);
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = mk(0.0, 0.0);
    }
    reduce_lanes8(acc, lane);
    double red[1] = {0.0};
    if (act && !(lane & 1)) {
        const int spin = ((lane >> 2) << 1) | ((lane >> 1) & 1), chi = spin >> 1;
        const double *cf = a.coef;
        const cx<double> d = mk(cf ? __ldg(cf + 4 + 2 * chi) : a.cd[chi][0], cf ? __ldg(cf + 5 + 2 * chi) : a.cd[chi][1]);
        const cx<double> cy = mk(cf ? __ldg(cf + 2 * chi) : a.cy[chi][0], cf ? __ldg(cf + 1 + 2 * chi) : a.cy[chi][1]);
        double2 *o = static_cast<double2 *>(a.out[p].data);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int plane = 3 * spin + k;
            cx<double> v = acc[k];
            if (kEpi == EPI_REAL_D) {
                v = d.re * v;
            } else if (kEpi == EPI_CPLX_D) {
                v = cmul(d, v);
            } else if (kEpi == EPI_REAL_YD || kEpi == EPI_CPLX_YD) {
                const double2 y = __ldg(static_cast<const double2 *>(a.y[p].data) + (size_t)plane * a.y[p].stride + i);
                if (kEpi == EPI_REAL_YD)
                    v = mk(fma(d.re, v.re, cy.re * y.x), fma(d.re, v.im, cy.re * y.y));
                else
                    v = cmac(cmul(cy, mk(y.x, y.y)), d, v);
            }
            o[(size_t)plane * a.out[p].stride + i] = make_double2(v.re, v.im);
            if (kReduce) red[0] += v.re * v.re + v.im * v.im;
        }
    }
    if (kReduce) grid_reduce_rhs<1>(red, 0, a.red, a.fin, a.state, a.red_out);
}

template <typename SF, typename GF, int D, int TPB>
cudaError_t launch_dslash_tpb(const DslashLaunch &a, cudaStream_t s)
{
    if (a.split == 8) {
        if constexpr (std::is_same<SF, SpF64>::value && GF::kRecon_ == 18) {
            if (a.rhs_log2 != 0) return cudaErrorInvalidValue;
            const dim3 grid(((8 * a.g.h + 127) / 128) * (a.both ? 2 : 1)), block(128);
#define QCD_DSL8(E, RD)                                                   \
    if (a.epi == E && a.reduce == RD) {                                   \
        dslash_lanes8_kernel<D, E, RD><<<grid, block, 0, s>>>(a);         \
        return cudaGetLastError();                                        \
    }
            QCD_DSL8(EPI_PLAIN, false)
            QCD_DSL8(EPI_CPLX_D, false)
            QCD_DSL8(EPI_REAL_YD, false)
            QCD_DSL8(EPI_REAL_YD, true)
            QCD_DSL8(EPI_CPLX_YD, false)
            QCD_DSL8(EPI_CPLX_YD, true)
#undef QCD_DSL8
        }
        return cudaErrorInvalidValue;
    }
    const dim3 grid((((a.g.h << a.rhs_log2) + TPB - 1) / TPB) * (a.both ? 2 : 1)), block(TPB);
#define QCD_DSL(E, RD)                                                      \
    if (a.epi == E && a.reduce == RD) {                                     \
        dslash_kernel<SF, GF, D, E, RD, TPB><<<grid, block, 0, s>>>(a);     \
        return cudaGetLastError();                                          \
    }
    QCD_DSL(EPI_PLAIN, false)
    QCD_DSL(EPI_CPLX_D, false)
    QCD_DSL(EPI_REAL_YD, false)
    QCD_DSL(EPI_REAL_YD, true)
    QCD_DSL(EPI_CPLX_YD, false)
    QCD_DSL(EPI_CPLX_YD, true)
#undef QCD_DSL
    return cudaErrorInvalidValue;
}

// Block sizes: the FP64-family kernels (~170 registers) always use 64; the
// FP32 / 16-bit ones take a.tpb in {64, 128, 256} (chosen by the autotuner,
// 128 by default).
template <typename SF, typename GF, int D>
cudaError_t launch_dslash_dag(const DslashLaunch &a, cudaStream_t s)
{
    if (sizeof(typename SF::R) == 8) return launch_dslash_tpb<SF, GF, D, 64>(a, s);  // (also the 8-lane FP64 kernel)
    if constexpr (sizeof(typename SF::R) != 8) {
        if (a.tpb == 64) return launch_dslash_tpb<SF, GF, D, 64>(a, s);
        if (a.tpb == 256) return launch_dslash_tpb<SF, GF, D, 256>(a, s);
        return launch_dslash_tpb<SF, GF, D, 128>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <typename SF, typename GF>
cudaError_t launch_dslash_fmt(const DslashLaunch &a, cudaStream_t s)
{
    return a.dagger ? launch_dslash_dag<SF, GF, 1>(a, s) : launch_dslash_dag<SF, GF, 0>(a, s);
}

}  // namespace qcd
