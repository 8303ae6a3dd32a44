// The hop of the 16-bit and FP32 hopping kernels in packed FP32 arithmetic.
//
// The two spin components of a half spinor are multiplied by the same link,
// so they form the two lanes of an FP32 pair: every multiply-add of the
// SU(3) product, of the spin projection and of the accumulation of the upper
// spins acts on both spins at once (one fma.rn.f32x2 instead of two FMAs).
// The operation is the one of dslash_kernel.cuh (the Wilson hop of CL2QCD,
// arXiv:1411.5219, Sec. 1): h = psi_up - S B psi_dn projected, U h or
// U^dagger h, lower spins rebuilt as -S B^dagger (U h), with the chiral
// basis gamma_mu = [[0, B], [B^dagger, 0]].
//
// Pair layout: lane 0 holds spin 0 (upper) or spin 2 (lower), lane 1 spin 1
// or spin 3.  Real and imaginary parts are kept in separate pairs.
#pragma once

#include "qcd_internal.cuh"

namespace qcd {

template <typename SF>
struct is_sp16 : std::false_type {};
template <typename H, bool N>
struct is_sp16<Sp16<H, N>> : std::true_type {};

// Formats whose hop runs in packed FP32 pairs (16-bit and FP32 spinors).
template <typename SF>
struct uses_pairs : is_sp16<SF> {};
template <>
struct uses_pairs<SpF32> : std::true_type {};

__device__ __forceinline__ float2 bc(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }

// 16-bit (re, im) word -> FP32 parts
template <typename H>
struct Half16Parts;
template <>
struct Half16Parts<__half> {
    __device__ __forceinline__ static float re(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
    __device__ __forceinline__ static float im(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
};
template <>
struct Half16Parts<__nv_bfloat16> {
    __device__ __forceinline__ static float re(uint32_t w) { return __uint_as_float(w << 16); }
    __device__ __forceinline__ static float im(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
};

// Half spinor in pairs: hr[c] = (Re h0_c, Re h1_c), hi[c] = (Im h0_c, Im h1_c).
struct HalfPairs {
    float2 r[3], i[3];
};

// Accumulated spinor in pairs: u* = spins (0, 1), l* = spins (2, 3).
struct AccPairs {
    float2 ur[3], ui[3], lr[3], li[3];
};

template <typename H>
__device__ __forceinline__ uint32_t word16(const uint4 (&w)[3], int k)
{
    const uint4 &p = w[k >> 2];
    return (k & 3) == 0 ? p.x : (k & 3) == 1 ? p.y : (k & 3) == 2 ? p.z : p.w;
}

// FP32 parts of spinor component k = 3 spin + colour of a fetched site.
template <typename SF>
struct PairSrc;
template <typename H, bool N>
struct PairSrc<Sp16<H, N>> {
    using Raw = typename Sp16<H, N>::Raw;
    __device__ __forceinline__ static float re(const Raw &r, int k) { return Half16Parts<H>::re(word16<H>(r.w, k)); }
    __device__ __forceinline__ static float im(const Raw &r, int k) { return Half16Parts<H>::im(word16<H>(r.w, k)); }
};
template <>
struct PairSrc<SpF32> {
    using Raw = SpF32::Raw;  // component k in float4 k / 2, (x, y) or (z, w)
    __device__ __forceinline__ static float re(const Raw &r, int k) { return k & 1 ? r.d[k >> 1].z : r.d[k >> 1].x; }
    __device__ __forceinline__ static float im(const Raw &r, int k) { return k & 1 ? r.d[k >> 1].w : r.d[k >> 1].y; }
};

// Spin projection of a fetched spinor (16-bit ones unscaled) straight from
// its storage: lane 0 is h_0 = psi_0 + ..., lane 1 is h_1 = psi_1 + ...; the
// lower spins enter in the order (3, 2) for x and y, (2, 3) for z and t.
template <typename SF>
struct is_fp16_spinor : std::false_type {};
template <bool N>
struct is_fp16_spinor<Sp16<__half, N>> : std::true_type {};

__device__ __forceinline__ __half2 as_h2(uint32_t w) { return *reinterpret_cast<__half2 *>(&w); }

// Packed 16-bit arithmetic on 32-bit words holding one complex number
// (re in the low half, im in the high half), for FP16 and BF16, and the
// mixed-precision FMA of sm_100+ (16-bit x 16-bit product, exact in FP32,
// added to an FP32 value).
template <typename H>
struct Word16;
template <>
struct Word16<__half> {
    __device__ __forceinline__ static uint32_t fma2(uint32_t a, uint32_t b, uint32_t c)
    {
        const __half2 d = __hfma2(*reinterpret_cast<__half2 *>(&a), *reinterpret_cast<__half2 *>(&b),
                                  *reinterpret_cast<__half2 *>(&c));
        return *reinterpret_cast<const uint32_t *>(&d);
    }
    __device__ __forceinline__ static uint32_t pack(float lo, float hi)
    {
        const __half2 d = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&d);
    }
    __device__ __forceinline__ static float fma(unsigned short a, unsigned short b, float c)
    {
        float d;
        asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(a), "h"(b), "f"(c));
        return d;
    }
};
template <>
struct Word16<__nv_bfloat16> {
    __device__ __forceinline__ static uint32_t fma2(uint32_t a, uint32_t b, uint32_t c)
    {
        const __nv_bfloat162 d = __hfma2(*reinterpret_cast<__nv_bfloat162 *>(&a),
                                         *reinterpret_cast<__nv_bfloat162 *>(&b),
                                         *reinterpret_cast<__nv_bfloat162 *>(&c));
        return *reinterpret_cast<const uint32_t *>(&d);
    }
    __device__ __forceinline__ static uint32_t pack(float lo, float hi)
    {
        const __nv_bfloat162 d = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&d);
    }
    __device__ __forceinline__ static float fma(unsigned short a, unsigned short b, float c)
    {
        float d;
        asm("fma.rn.f32.bf16 %0, %1, %2, %3;" : "=f"(d) : "h"(a), "h"(b), "f"(c));
        return d;
    }
};
__device__ __forceinline__ uint32_t swap_halves(uint32_t w) { return __byte_perm(w, 0, 0x1032); }
// sign flips as integer operations (off the FMA pipe)
__device__ __forceinline__ uint32_t neg_im(uint32_t w) { return w ^ 0x80000000u; }
__device__ __forceinline__ uint32_t neg_re(uint32_t w) { return w ^ 0x00008000u; }
__device__ __forceinline__ uint32_t neg_both(uint32_t w) { return w ^ 0x80008000u; }

// 16-bit spinors: the spin projection in packed 16-bit arithmetic on the
// stored (re, im) words: hw[s][c] = h_s of colour c as such a word.  h is
// rounded to the 16-bit format once more (half a unit of |h|, within the
// storage tolerance).
template <typename SF, int MU, int S>
__device__ __forceinline__ void project_words(const typename SF::Raw &w, uint32_t (&hw)[2][3])
{
    using H = typename SF::H16;
    using W = Word16<H>;
    constexpr int b0 = MU <= 1 ? 3 : 2, b1 = MU <= 1 ? 2 : 3;
    constexpr float s = (float)S;
    const uint32_t pp = W::pack(s, s), mm = W::pack(-s, -s), mp = W::pack(-s, s), pm = W::pack(s, -s);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const uint32_t a0 = word16<H>(w.w, c), a1 = word16<H>(w.w, 3 + c);
        const uint32_t x0 = word16<H>(w.w, 3 * b0 + c), x1 = word16<H>(w.w, 3 * b1 + c);
        if (MU == 0) {  // (psi0 + S i psi3, psi1 + S i psi2); i z = (-im, re)
            hw[0][c] = W::fma2(swap_halves(x0), mp, a0);
            hw[1][c] = W::fma2(swap_halves(x1), mp, a1);
        } else if (MU == 1) {  // (psi0 + S psi3, psi1 - S psi2)
            hw[0][c] = W::fma2(x0, pp, a0);
            hw[1][c] = W::fma2(x1, mm, a1);
        } else if (MU == 2) {  // (psi0 + S i psi2, psi1 - S i psi3)
            hw[0][c] = W::fma2(swap_halves(x0), mp, a0);
            hw[1][c] = W::fma2(swap_halves(x1), pm, a1);
        } else {  // (psi0 - S psi2, psi1 - S psi3)
            hw[0][c] = W::fma2(x0, mm, a0);
            hw[1][c] = W::fma2(x1, mm, a1);
        }
    }
}

template <typename SF, int MU, int S>
__device__ __forceinline__ HalfPairs project_pairs(const typename SF::Raw &w)
{
    using P = PairSrc<SF>;
    constexpr int b0 = MU <= 1 ? 3 : 2, b1 = MU <= 1 ? 2 : 3;
    constexpr float s = (float)S;
    HalfPairs h;
    if constexpr (is_fp16_spinor<SF>::value) {
        // 12 conversions to FP32 instead of 24 (they run on the FMA pipe)
        uint32_t hw[2][3];
        project_words<SF, MU, S>(w, hw);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 f0 = __half22float2(as_h2(hw[0][c])), f1 = __half22float2(as_h2(hw[1][c]));
            h.r[c] = make_float2(f0.x, f1.x);
            h.i[c] = make_float2(f0.y, f1.y);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int a0 = c, a1 = 3 + c, x0 = 3 * b0 + c, x1 = 3 * b1 + c;
            const float2 ar = make_float2(P::re(w, a0), P::re(w, a1)), ai = make_float2(P::im(w, a0), P::im(w, a1));
            const float2 xr = make_float2(P::re(w, x0), P::re(w, x1)), xi = make_float2(P::im(w, x0), P::im(w, x1));
            if (MU == 0) {  // h = (psi0 + S i psi3, psi1 + S i psi2)
                h.r[c] = fma2(xi, make_float2(-s, -s), ar);
                h.i[c] = fma2(xr, make_float2(s, s), ai);
            } else if (MU == 1) {  // h = (psi0 + S psi3, psi1 - S psi2)
                h.r[c] = fma2(xr, make_float2(s, -s), ar);
                h.i[c] = fma2(xi, make_float2(s, -s), ai);
            } else if (MU == 2) {  // h = (psi0 + S i psi2, psi1 - S i psi3)
                h.r[c] = fma2(xi, make_float2(-s, s), ar);
                h.i[c] = fma2(xr, make_float2(s, -s), ai);
            } else {  // h = (psi0 - S psi2, psi1 - S psi3)
                h.r[c] = fma2(xr, make_float2(-s, -s), ar);
                h.i[c] = fma2(xi, make_float2(-s, -s), ai);
            }
        }
    }
    return h;
}

// U h (kAdj false) or U^dagger h (kAdj true) on both spins.
template <bool kAdj>
__device__ __forceinline__ HalfPairs su3_pairs(const Link<float> &u, const HalfPairs &h)
{
    const float2 m1 = make_float2(-1.0f, -1.0f);
    HalfPairs v;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!kAdj) {
            // Re = sum Re U Re h - Im U Im h ; Im = sum Re U Im h + Im U Re h
            float2 p = mul2(bc(u.m[a][0].re), h.r[0]);
            float2 q = mul2(bc(u.m[a][0].im), h.i[0]);
            float2 t = mul2(bc(u.m[a][0].re), h.i[0]);
            t = fma2(bc(u.m[a][0].im), h.r[0], t);
#pragma unroll
            for (int j = 1; j < 3; ++j) {
                p = fma2(bc(u.m[a][j].re), h.r[j], p);
                q = fma2(bc(u.m[a][j].im), h.i[j], q);
                t = fma2(bc(u.m[a][j].re), h.i[j], t);
                t = fma2(bc(u.m[a][j].im), h.r[j], t);
            }
            v.r[a] = fma2(q, m1, p);
            v.i[a] = t;
        } else {
            // Re = sum Re U_ja Re h + Im U_ja Im h ; Im = sum Re U_ja Im h - Im U_ja Re h
            float2 t = mul2(bc(u.m[0][a].re), h.r[0]);
            t = fma2(bc(u.m[0][a].im), h.i[0], t);
            float2 p = mul2(bc(u.m[0][a].re), h.i[0]);
            float2 q = mul2(bc(u.m[0][a].im), h.r[0]);
#pragma unroll
            for (int j = 1; j < 3; ++j) {
                t = fma2(bc(u.m[j][a].re), h.r[j], t);
                t = fma2(bc(u.m[j][a].im), h.i[j], t);
                p = fma2(bc(u.m[j][a].re), h.i[j], p);
                q = fma2(bc(u.m[j][a].im), h.r[j], q);
            }
            v.r[a] = t;
            v.i[a] = fma2(q, m1, p);
        }
    }
    return v;
}

// acc (+)= w * (the full spinor rebuilt from v): upper = v, lower =
// -S B^dagger v.  In pairs the lower spins of x and y take v with its lanes
// swapped (spin 2 gains from spin 1 and spin 3 from spin 0).
template <int MU, int S, bool kFirst>
__device__ __forceinline__ void accumulate_pairs(AccPairs &acc, const HalfPairs &v, float w)
{
    const float ws = w * (float)S;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 lr_w, li_w, lr_v, li_v;  // lower += lr_w * lr_v (real), li_w * li_v (imag)
        if (MU == 0) {  // (l2, l3) = -S (i u1, i u0)
            lr_v = swp(v.i[c]);
            lr_w = bc(ws);
            li_v = swp(v.r[c]);
            li_w = bc(-ws);
        } else if (MU == 1) {  // (l2, l3) = -S (u1, -u0)
            lr_v = swp(v.r[c]);
            li_v = swp(v.i[c]);
            lr_w = li_w = make_float2(-ws, ws);
        } else if (MU == 2) {  // (l2, l3) = -S (i u0, -i u1)
            lr_v = v.i[c];
            lr_w = make_float2(ws, -ws);
            li_v = v.r[c];
            li_w = make_float2(-ws, ws);
        } else {  // (l2, l3) = -S (u0, u1)
            lr_v = v.r[c];
            li_v = v.i[c];
            lr_w = li_w = bc(-ws);
        }
        if (kFirst) {
            acc.ur[c] = mul2(bc(w), v.r[c]);
            acc.ui[c] = mul2(bc(w), v.i[c]);
            acc.lr[c] = mul2(lr_w, lr_v);
            acc.li[c] = mul2(li_w, li_v);
        } else {
            acc.ur[c] = fma2(bc(w), v.r[c], acc.ur[c]);
            acc.ui[c] = fma2(bc(w), v.i[c], acc.ui[c]);
            acc.lr[c] = fma2(lr_w, lr_v, acc.lr[c]);
            acc.li[c] = fma2(li_w, li_v, acc.li[c]);
        }
    }
}

// ---- 16-bit spinors with links of the same 16-bit format (reconstruct 12
// or 18): the SU(3) product by mixed-precision FMA straight from the stored
// link words and the packed-projected half spinor, so neither needs
// converting to FP32 and no link entry is copied into both lanes of a pair.
// Measured on GB300: fma.rn.f32.f16 issues at the FFMA rate, and with
// operands taken from the halves of 32-bit words it ran 25 % above
// conversions plus packed FMAs.

template <typename SF, typename GF>
struct is_mixed16 : std::false_type {};
template <typename H, bool N>
struct is_mixed16<Sp16<H, N>, G16<H, 12>> : std::true_type {};
template <typename H, bool N>
struct is_mixed16<Sp16<H, N>, G16<H, 18>> : std::true_type {};

// the (re, im) halves of a word as 16-bit registers
__device__ __forceinline__ void halves(uint32_t w, unsigned short &re, unsigned short &im)
{
    asm("mov.b32 {%0, %1}, %2;" : "=h"(re), "=h"(im) : "r"(w));
}

// U (kAdj false) or U^dagger (kAdj true) times the two half-spinor spins,
// from the link's words (u[row][col]), into FP32 pairs.
template <typename H, bool kAdj>
__device__ __forceinline__ HalfPairs su3_mixed(const uint32_t (&u)[3][3], const uint32_t (&hw)[2][3])
{
    using W = Word16<H>;
    // re and im halves of h, and of h with one part negated (the minus signs
    // of the complex products)
    unsigned short hr[2][3], hi[2][3], hn[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            unsigned short r_, i_, nr_, ni_;
            halves(hw[s][b], r_, i_);
            halves(kAdj ? neg_re(hw[s][b]) : neg_im(hw[s][b]), nr_, ni_);
            hr[s][b] = r_;
            hi[s][b] = i_;
            hn[s][b] = kAdj ? nr_ : ni_;  // -Re h (adjoint) or -Im h
        }
    HalfPairs v;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float re[2], im[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            float r_ = 0.0f, i_ = 0.0f;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                unsigned short ur, ui;
                halves(kAdj ? u[b][a] : u[a][b], ur, ui);
                if (!kAdj) {  // Re += ur hr - ui hi ; Im += ur hi + ui hr
                    r_ = W::fma(ur, hr[s][b], r_);
                    r_ = W::fma(ui, hn[s][b], r_);
                    i_ = W::fma(ur, hi[s][b], i_);
                    i_ = W::fma(ui, hr[s][b], i_);
                } else {  // conj(U_ba) h: Re += ur hr + ui hi ; Im += ur hi - ui hr
                    r_ = W::fma(ur, hr[s][b], r_);
                    r_ = W::fma(ui, hi[s][b], r_);
                    i_ = W::fma(ur, hi[s][b], i_);
                    i_ = W::fma(ui, hn[s][b], i_);
                }
            }
            re[s] = r_;
            im[s] = i_;
        }
        v.r[a] = make_float2(re[0], re[1]);
        v.i[a] = make_float2(im[0], im[1]);
    }
    return v;
}

// The link as words; reconstruct-12 rebuilds row 2 = conj(row 0 x row 1)
// from the stored rows with exact products and FP32 sums, and rounds it to
// the 16-bit format (half a unit per entry).
template <typename H, int kRecon>
__device__ __forceinline__ void link_words(const typename G16<H, kRecon>::Raw &r, uint32_t (&u)[3][3])
{
    using W = Word16<H>;
#pragma unroll
    for (int k = 0; k < kRecon / 2; ++k) u[k / 3][k % 3] = r.w[k];
    if constexpr (kRecon == 12) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int a = (c + 1) % 3, b = (c + 2) % 3;
            // P = U0a U1b - U0b U1a ; row 2 = conj(P)
            unsigned short ar, ai, br, bi, cr, ci, dr, di, nar, nai, ncr, nci;
            halves(u[0][a], ar, ai);
            halves(u[1][b], br, bi);
            halves(u[0][b], cr, ci);
            halves(u[1][a], dr, di);
            halves(neg_both(u[0][a]), nar, nai);
            halves(neg_both(u[0][b]), ncr, nci);
            // Re P = ar br - ai bi - cr dr + ci di
            float re = W::fma(ar, br, 0.0f);
            re = W::fma(nai, bi, re);
            re = W::fma(ncr, dr, re);
            re = W::fma(ci, di, re);
            // -Im P = -(ar bi + ai br) + cr di + ci dr
            float mi = W::fma(nar, bi, 0.0f);
            mi = W::fma(nai, br, mi);
            mi = W::fma(cr, di, mi);
            mi = W::fma(ci, dr, mi);
            u[2][c] = W::pack(re, mi);
        }
    }
}

// One hop of a 16-bit spinor: project, multiply, rebuild and accumulate;
// `flip` applies the boundary factor -1 (folded into the weight with the
// FP16 per-site scale).
template <typename SF, typename GF, int MU, int S, bool kAdj, bool kFirst>
__device__ __forceinline__ void hop_pairs(AccPairs &acc, const typename SF::Raw &rs, const typename GF::Raw &ru,
                                          bool flip)
{
    HalfPairs v;
    if constexpr (is_mixed16<SF, GF>::value) {
        using H = typename SF::H16;
        uint32_t hw[2][3], u[3][3];
        project_words<SF, MU, S>(rs, hw);
        link_words<H, GF::kRecon_>(ru, u);
        v = su3_mixed<H, kAdj>(u, hw);
    } else {
        const HalfPairs h = project_pairs<SF, MU, S>(rs);
        v = su3_pairs<kAdj>(GF::decode(ru), h);
    }
    const float sc = SF::scale(rs);
    accumulate_pairs<MU, S, kFirst>(acc, v, flip ? -sc : sc);
}

__device__ __forceinline__ Spinor<float> unpair(const AccPairs &a)
{
    Spinor<float> s;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s.c[0][c] = mk(a.ur[c].x, a.ui[c].x);
        s.c[1][c] = mk(a.ur[c].y, a.ui[c].y);
        s.c[2][c] = mk(a.lr[c].x, a.li[c].x);
        s.c[3][c] = mk(a.lr[c].y, a.li[c].y);
    }
    return s;
}

}  // namespace qcd
