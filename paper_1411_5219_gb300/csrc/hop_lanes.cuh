// One hop per thread, eight threads per site, FP64 (reconstruct-18 links).
//
// An FP64 warp instruction holds its sub-partition's FP64 unit for 64 cycles
// on GB300, so a thread that does all eight hops of a site (~790 FP64
// instructions) needs >= 24 us however empty the GPU is.  On small lattices
// that latency, not throughput, sets the time.  Here eight adjacent lanes
// take the eight hops of one site (k = 2 mu + backward) and sum their
// partial spinors with shuffles.  The spin projection and the lower-spin
// rebuild of the chiral basis are table-driven (one nonzero +-1 or +-i per
// row of B_mu), so they are lane selections and sign flips: no FP64
// arithmetic and no branches on the direction.  The operation is the Wilson
// hop of CL2QCD (arXiv:1411.5219, Sec. 1): (1 - S gamma_mu) U_mu(x)
// psi(x+mu) forward, (1 + S gamma_mu) U_mu(x-mu)^dagger psi(x-mu) backward,
// S = -1 for the adjoint.
#pragma once

#include "qcd_internal.cuh"

namespace qcd {

// ---- spin algebra of one hop, table-driven.  gamma_mu = [[0, B], [B^dag, 0]]:
// B_0 = -i sigma_1, B_1 = -i sigma_2, B_2 = -i sigma_3, B_3 = 1.  Row s of B
// has one nonzero entry, in column perm(s) (swap for x and y, identity for z
// and t), with value in {+-1, +-i}: coded as (is_imag, negative).
__device__ __forceinline__ void b_entry(int mu, int s, int &col, bool &imag, bool &neg)
{
    col = mu <= 1 ? 1 - s : s;
    imag = mu == 0 || mu == 2;
    // B_0: -i, -i ; B_1: -1 (row 0), +1 (row 1) ; B_2: -i, +i ; B_3: +1, +1
    neg = mu == 0 ? true : mu == 1 ? (s == 0) : mu == 2 ? (s == 0) : false;
}

__device__ __forceinline__ double flip_sign(double v, bool neg)
{
    return __longlong_as_double(__double_as_longlong(v) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
}

// (c * z) for c in {+-1, +-i}: a selection of parts and signs, no FP64 arithmetic.
__device__ __forceinline__ cx<double> unit_mul(cx<double> z, bool imag, bool neg)
{
    cx<double> r = imag ? cx<double>{-z.im, z.re} : z;
    return {flip_sign(r.re, neg), flip_sign(r.im, neg)};
}

// The 24 doubles (12 complex, index 3 spin + colour) that hop k of site i
// (parity p of the output) contributes to (D psi)(x): k = 2 mu + (backward).
// U: FP64 reconstruct-18 links, block (parity * 4 + mu) of 9 double2
// planes; in: the 12 double2 planes of the input half field.  kCoherent:
// the input was written earlier in the same kernel launch (read through
// L2, not the non-coherent read-only path).
template <bool kCoherent>
__device__ __forceinline__ void hop_lane8(const Geom &g, const double2 *U, int ustride, const double2 *ind,
                                          int instride, int p, int i, int k, bool dagger, cx<double> (&acc)[12])
{
    const SiteCoords c = site_coords(g, i, p);
    const int mu = k >> 1;
    const bool bwd = k & 1;
    int nb;
    bool flip = false;
    if (mu == 0) {
        const int xn = bwd ? (c.x == 0 ? g.L[0] - 1 : c.x - 1) : (c.x + 1 == g.L[0] ? 0 : c.x + 1);
        nb = i - c.xh + (xn >> 1);
    } else {
        const int L = g.L[mu];
        const int st = mu == 1 ? g.sy : mu == 2 ? g.sz : g.st;
        const int x = mu == 1 ? c.y : mu == 2 ? c.z : c.t;
        const bool wrap = bwd ? x == 0 : x == L - 1;
        nb = wrap ? (bwd ? i + (L - 1) * st : i - (L - 1) * st) : (bwd ? i - st : i + st);
        flip = mu == 3 && wrap && antiperiodic(g);
    }
    // the neighbour spinor
    cx<double> psi[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        const double2 v = kCoherent ? __ldcg(ind + (size_t)a * instride + nb) : __ldg(ind + (size_t)a * instride + nb);
        psi[a] = mk(v.x, v.y);
    }
    // the link: forward U_mu(x) (block (p, mu), this site), backward
    // U_mu(x - mu)^dagger (block (1 - p, mu), the neighbour)
    const int blk = (bwd ? 1 - p : p) * 4 + mu, li = bwd ? nb : i;
    const double2 *up = U + (size_t)blk * 9 * ustride + li;
    cx<double> m[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const double2 v = __ldg(up + (size_t)(bwd ? 3 * b + a : 3 * a + b) * ustride);
            m[a][b] = bwd ? mk(v.x, -v.y) : mk(v.x, v.y);
        }
    // projector sign: (1 - S gamma) forward, (1 + S gamma) backward; S = -1
    // for D^dagger (a negative product when exactly one of the two holds)
    const bool sneg = dagger != bwd;
    // h_s = psi_s - S B[s][col] psi_{2 + col}
    cx<double> h[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        int col;
        bool imag, neg;
        b_entry(mu, s, col, imag, neg);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const cx<double> z = unit_mul(col ? psi[9 + a] : psi[6 + a], imag, !(neg ^ sneg));  // -S B z
            h[s][a] = psi[3 * s + a] + z;
        }
    }
    // u = m h on both spins
    cx<double> u[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<double> v = cmul(m[a][0], h[s][0]);
            v = cmac(v, m[a][1], h[s][1]);
            v = cmac(v, m[a][2], h[s][2]);
            u[s][a] = v;
        }
    // upper spins: u; lower spin t: -S conj(B[col][t]) u_col (col = perm(t));
    // the boundary factor -1 on the wrapping t hop
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[3 * s + a] = {flip_sign(u[s][a].re, flip), flip_sign(u[s][a].im, flip)};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        int col;
        bool imag, neg;
        b_entry(mu, t, col, imag, neg);  // perm is an involution: B[col][t] has the same kind
        int c2;
        bool imag2, neg2;
        b_entry(mu, col, c2, imag2, neg2);
        // conj(B[col][t]): an imaginary entry changes sign
        const bool cneg = imag2 ? !neg2 : neg2;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const cx<double> z = unit_mul(col ? u[1][a] : u[0][a], imag2, !(cneg ^ sneg) ^ flip);
            acc[3 * (2 + t) + a] = z;
        }
    }
}

// Sum of the eight lanes' partial spinors of a site: afterwards the lanes
// with bit 0 clear hold, in acc[0..2], the three colours of spin
// 2 (lane >> 2) + ((lane >> 1) & 1).  Every lane of the warp must call it.
__device__ __forceinline__ void reduce_lanes8(cx<double> (&acc)[12], int lane)
{
    // lanes with bit 2 clear keep the upper spins, then bit 1 picks the spin,
    // then the pair adds all
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        const bool up = !(lane & 4);
        const cx<double> keep = up ? acc[a] : acc[6 + a], give = up ? acc[6 + a] : acc[a];
        const double gr = __shfl_xor_sync(0xffffffffu, give.re, 4), gi = __shfl_xor_sync(0xffffffffu, give.im, 4);
        acc[a] = mk(keep.re + gr, keep.im + gi);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const bool first = !(lane & 2);
        const cx<double> keep = first ? acc[a] : acc[3 + a], give = first ? acc[3 + a] : acc[a];
        const double gr = __shfl_xor_sync(0xffffffffu, give.re, 2), gi = __shfl_xor_sync(0xffffffffu, give.im, 2);
        acc[a] = mk(keep.re + gr, keep.im + gi);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double gr = __shfl_xor_sync(0xffffffffu, acc[a].re, 1), gi = __shfl_xor_sync(0xffffffffu, acc[a].im, 1);
        acc[a] = mk(acc[a].re + gr, acc[a].im + gi);
    }
}

}  // namespace qcd
