// Internal definitions shared by the libqcd CUDA translation units:
// complex arithmetic, device storage formats of spinor and gauge fields,
// lattice geometry with even-odd indexing, deterministic block reductions
// and the device-resident CG state.
//
// Conventions (the paper, CL2QCD arXiv:1411.5219, names the Wilson and
// twisted-mass Wilson matrices in Sec. 3 but prints no formulas; these are
// the standard ones):
//   D_hop psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
//                       + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu)
//   chiral basis: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 =
//   [[0, 1], [1, 0]], gamma_5 = diag(1, 1, -1, -1); the t-hop that wraps the
//   lattice carries the factor t_bc (-1 antiperiodic).
//   Sites: lex = x + Lx (y + Ly (z + Lz t)), parity (x+y+z+t) mod 2, index
//   within a parity lex/2.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/qcd.h"
#include "df64.cuh"

namespace qcd {

// ------------------------------------------------------------------ complex

template <typename R>
struct cx {
    R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
// conj(a) * b
template <typename R>
__device__ __forceinline__ cx<R> cjmul(cx<R> a, cx<R> b) { return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re}; }
// acc + a * b
template <typename R>
__device__ __forceinline__ cx<R> cmac(cx<R> acc, cx<R> a, cx<R> b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
    return acc;
}
// acc + conj(a) * b
template <typename R>
__device__ __forceinline__ cx<R> cjmac(cx<R> acc, cx<R> a, cx<R> b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
    return acc;
}
// i * a
template <typename R>
__device__ __forceinline__ cx<R> ti(cx<R> a) { return {-a.im, a.re}; }
template <typename R>
__device__ __forceinline__ cx<R> conjg(cx<R> a) { return {a.re, -a.im}; }

template <typename R>
struct Spinor {
    cx<R> c[4][3];
};
template <typename R>
struct HalfSpinor {
    cx<R> c[2][3];
};
template <typename R>
struct Link {
    cx<R> m[3][3];
};

// ------------------------------------------------------------------ storage
//
// A half field (one parity, h sites) is stored as "planes": plane j holds
// vector element j of every site, site-fastest, so a warp reading one plane
// reads consecutive 8- or 16-byte words (structure of arrays; the paper's
// Sec. 4 stresses SoA for GPUs).  `stride` is the padded site count of a
// plane.  FP16 spinors carry one FP32 scale per site (the largest |real
// component| of the site); BF16 spinors and all 16-bit links are stored
// unscaled.

struct SpinorView {
    void *data;      // first plane
    float *norm;     // FP16 only: per-site scale, else nullptr
    int stride;      // sites per plane (padded)
};

struct GaugeView {
    void *data;      // block (parity, mu) = parity*4 + mu, planes inside each block
    int stride;      // sites per plane (padded)
};

// Spinor storage formats.  load() returns the full 4x3 spinor of site i in
// arithmetic precision R; store() writes it.
struct SpF64 {
    using R = double;
    static constexpr int kPlanes = 12;  // double2 per plane
    static constexpr size_t kBytesPerSite = 192;
    static constexpr bool kScaled = false;
    struct Raw {
        double2 d[12];
    };
    __device__ __forceinline__ static Raw fetch(const SpinorView &v, int i)
    {
        Raw r;
        const double2 *p = static_cast<const double2 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 12; ++k) r.d[k] = __ldg(p + (size_t)k * v.stride);
        return r;
    }
    __device__ __forceinline__ static Spinor<R> decode(const Raw &r)
    {
        Spinor<R> s;
#pragma unroll
        for (int k = 0; k < 12; ++k) s.c[k / 3][k % 3] = mk(r.d[k].x, r.d[k].y);
        return s;
    }
    __device__ __forceinline__ static R scale(const Raw &) { return 1.0; }
    __device__ __forceinline__ static Spinor<R> load(const SpinorView &v, int i)
    {
        Spinor<R> s;
        const double2 *p = static_cast<const double2 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 d = __ldg(p + (size_t)k * v.stride);
            s.c[k / 3][k % 3] = mk(d.x, d.y);
        }
        return s;
    }
    __device__ __forceinline__ static void store(const SpinorView &v, int i, const Spinor<R> &s)
    {
        double2 *p = static_cast<double2 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(size_t)k * v.stride] = make_double2(s.c[k / 3][k % 3].re, s.c[k / 3][k % 3].im);
    }
};

struct SpF32 {
    using R = float;
    static constexpr int kPlanes = 6;  // float4 (two complex) per plane
    static constexpr size_t kBytesPerSite = 96;
    static constexpr bool kScaled = false;
    struct Raw {
        float4 d[6];
    };
    __device__ __forceinline__ static Raw fetch(const SpinorView &v, int i)
    {
        Raw r;
        const float4 *p = static_cast<const float4 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 6; ++k) r.d[k] = __ldg(p + (size_t)k * v.stride);
        return r;
    }
    __device__ __forceinline__ static Spinor<R> decode(const Raw &r)
    {
        Spinor<R> s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            s.c[(2 * k) / 3][(2 * k) % 3] = mk(r.d[k].x, r.d[k].y);
            s.c[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(r.d[k].z, r.d[k].w);
        }
        return s;
    }
    __device__ __forceinline__ static R scale(const Raw &) { return 1.0f; }
    __device__ __forceinline__ static Spinor<R> load(const SpinorView &v, int i)
    {
        Spinor<R> s;
        const float4 *p = static_cast<const float4 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 d = __ldg(p + (size_t)k * v.stride);
            s.c[(2 * k) / 3][(2 * k) % 3] = mk(d.x, d.y);
            s.c[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(d.z, d.w);
        }
        return s;
    }
    __device__ __forceinline__ static void store(const SpinorView &v, int i, const Spinor<R> &s)
    {
        float4 *p = static_cast<float4 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const cx<R> a = s.c[(2 * k) / 3][(2 * k) % 3], b = s.c[(2 * k + 1) / 3][(2 * k + 1) % 3];
            p[(size_t)k * v.stride] = make_float4(a.re, a.im, b.re, b.im);
        }
    }
};

template <typename H>
struct Half16;
template <>
struct Half16<__half> {
    __device__ __forceinline__ static float2 to2(uint32_t w)
    {
        __half2 h = *reinterpret_cast<__half2 *>(&w);
        return __half22float2(h);
    }
    __device__ __forceinline__ static uint32_t from2(float a, float b)
    {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
};
template <>
struct Half16<__nv_bfloat16> {
    __device__ __forceinline__ static float2 to2(uint32_t w)
    {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&w);
        return __bfloat1622float2(h);
    }
    __device__ __forceinline__ static uint32_t from2(float a, float b)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
};

// Double-float spinor: twelve float4 planes, (hi.re, hi.im, lo.re, lo.im)
// per complex component, 192 bytes per site like FP64.
struct SpDF64 {
    using R = df;
    static constexpr int kPlanes = 12;
    static constexpr size_t kBytesPerSite = 192;
    static constexpr bool kScaled = false;
    struct Raw {
        float4 d[12];
    };
    __device__ __forceinline__ static Raw fetch(const SpinorView &v, int i)
    {
        Raw r;
        const float4 *p = static_cast<const float4 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 12; ++k) r.d[k] = __ldg(p + (size_t)k * v.stride);
        return r;
    }
    __device__ __forceinline__ static Spinor<R> decode(const Raw &r)
    {
        Spinor<R> s;
#pragma unroll
        for (int k = 0; k < 12; ++k) s.c[k / 3][k % 3] = cx<R>{df(r.d[k].x, r.d[k].z), df(r.d[k].y, r.d[k].w)};
        return s;
    }
    __device__ __forceinline__ static R scale(const Raw &) { return df(1.0f, 0.0f); }
    __device__ __forceinline__ static Spinor<R> load(const SpinorView &v, int i) { return decode(fetch(v, i)); }
    __device__ __forceinline__ static void store(const SpinorView &v, int i, const Spinor<R> &s)
    {
        float4 *p = static_cast<float4 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const cx<R> a = s.c[k / 3][k % 3];
            p[(size_t)k * v.stride] = make_float4(a.re.hi, a.im.hi, a.re.lo, a.im.lo);
        }
    }
};

// 16-bit spinor: three uint4 planes (four complex each); FP16 adds a scale.
template <typename H, bool kNorm>
struct Sp16 {
    using R = float;
    using H16 = H;
    static constexpr int kPlanes = 3;
    static constexpr size_t kBytesPerSite = 48 + (kNorm ? 4 : 0);
    // decode() leaves the FP16 per-site scale out; scale() returns it, so the
    // hopping kernel can fold it into its accumulation instead of scaling
    // all 24 components.
    static constexpr bool kScaled = kNorm;
    struct Raw {
        uint4 w[3];
        float sc;
    };
    __device__ __forceinline__ static Raw fetch(const SpinorView &v, int i)
    {
        Raw r;
        const uint4 *p = static_cast<const uint4 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) r.w[k] = __ldg(p + (size_t)k * v.stride);
        r.sc = kNorm ? __ldg(v.norm + i) : 1.0f;
        return r;
    }
    __device__ __forceinline__ static Spinor<R> decode(const Raw &r)
    {
        Spinor<R> s;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint32_t ws[4] = {r.w[k].x, r.w[k].y, r.w[k].z, r.w[k].w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 f = Half16<H>::to2(ws[j]);
                const int c = 4 * k + j;
                s.c[c / 3][c % 3] = mk(f.x, f.y);
            }
        }
        return s;
    }
    __device__ __forceinline__ static R scale(const Raw &r) { return r.sc; }
    __device__ __forceinline__ static Spinor<R> load(const SpinorView &v, int i)
    {
        Spinor<R> s;
        const uint4 *p = static_cast<const uint4 *>(v.data) + i;
        const float sc = kNorm ? __ldg(v.norm + i) : 1.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 w = __ldg(p + (size_t)k * v.stride);
            uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 f = Half16<H>::to2(ws[j]);
                const int c = 4 * k + j;
                s.c[c / 3][c % 3] = mk(sc * f.x, sc * f.y);
            }
        }
        return s;
    }
    __device__ __forceinline__ static void store(const SpinorView &v, int i, const Spinor<R> &s)
    {
        float inv = 1.0f;
        if (kNorm) {
            float m = 0.0f;
#pragma unroll
            for (int c = 0; c < 12; ++c) m = fmaxf(m, fmaxf(fabsf(s.c[c / 3][c % 3].re), fabsf(s.c[c / 3][c % 3].im)));
            v.norm[i] = m;
            inv = m > 0.0f ? 1.0f / m : 0.0f;
        }
        uint4 *p = static_cast<uint4 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint32_t ws[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = 4 * k + j;
                ws[j] = Half16<H>::from2(inv * s.c[c / 3][c % 3].re, inv * s.c[c / 3][c % 3].im);
            }
            p[(size_t)k * v.stride] = make_uint4(ws[0], ws[1], ws[2], ws[3]);
        }
    }
};
using SpF16 = Sp16<__half, true>;
using SpBF16 = Sp16<__nv_bfloat16, false>;

// Gauge storage formats: kRecon = 18 (full matrix), 12 (rows 0 and 1;
// row 2 = conj(row0 x row1), valid for SU(3)) or 8 (eight reals, below).
//
// Reconstruct-8, pivoted for links near the identity.  Work on W = U with
// its columns reversed (W_ij = U_i,2-j; unitary with det W = -1), so that
// the two entries recovered from a norm, w02 = U_00 and w20 = U_22, are the
// large diagonal ones and the divisor N = |w01|^2 + |w02|^2 is close to 1.
// Stored: w00, w01, w10 (complex) and the half-angle tangents t = tan(arg/2)
// of w02 and w20 (a phase e^{i arg} = ((1 - t^2) + 2 i t) / (1 + t^2), one
// division instead of sin and cos; the angular error stays below the storage
// rounding of t).  Rows a, b, c of W: |w02| and |w20| follow from the unit
// norm of row a and column 0; orthogonality of a and b together with
// c = -conj(a x b) (det W = -1) gives a 2x2 linear system for w11, w12 with
// determinant -N; the rest of row c is -conj(a x b).
template <typename R>
__host__ __device__ __forceinline__ R half_angle_tan(cx<R> w, R tmax)
{
    const R a = sqrt(w.re * w.re + w.im * w.im);
    if (!(a > R(0))) return R(0);
    R t;
    if (w.re >= R(0))
        t = w.im / (a + w.re);
    else
        t = w.im == R(0) ? tmax : (a - w.re) / w.im;
    return t > tmax ? tmax : (t < -tmax ? -tmax : t);
}

template <typename R>
__host__ __device__ __forceinline__ void recon8_encode(const Link<R> &u, R p[8], R tmax)
{
    // W = U with reversed columns
    const cx<R> w00 = u.m[0][2], w01 = u.m[0][1], w02 = u.m[0][0], w10 = u.m[1][2], w20 = u.m[2][2];
    p[0] = w00.re;
    p[1] = w00.im;
    p[2] = w01.re;
    p[3] = w01.im;
    p[4] = w10.re;
    p[5] = w10.im;
    p[6] = half_angle_tan(w02, tmax);
    p[7] = half_angle_tan(w20, tmax);
}

template <typename R>
__host__ __device__ __forceinline__ cx<R> unit_phase(R t)
{
    const R r = R(1) / (R(1) + t * t);
    return {(R(1) - t * t) * r, R(2) * t * r};
}

template <typename R>
__device__ __forceinline__ Link<R> recon8_decode(const R p[8])
{
    const cx<R> w00 = mk(p[0], p[1]), w01 = mk(p[2], p[3]), w10 = mk(p[4], p[5]);
    const R n00 = w00.re * w00.re + w00.im * w00.im;
    const R n01 = w01.re * w01.re + w01.im * w01.im;
    const R n10 = w10.re * w10.re + w10.im * w10.im;
    const R r02 = R(1) - n00 - n01, r20 = R(1) - n00 - n10;
    const R a02 = sqrt(r02 > R(0) ? r02 : R(0)), a20 = sqrt(r20 > R(0) ? r20 : R(0));
    const cx<R> w02 = a02 * unit_phase(p[6]), w20 = a20 * unit_phase(p[7]);
    const R inv_n = R(1) / (n01 + a02 * a02);
    const cx<R> w11 = inv_n * (cmul(conjg(w20), conjg(w02)) - cmul(cmul(w01, conjg(w00)), w10));
    const cx<R> w12 = -(inv_n * (cmul(cmul(w02, conjg(w00)), w10) + cmul(conjg(w01), conjg(w20))));
    const cx<R> w21 = -conjg(cmul(w02, w10) - cmul(w00, w12));
    const cx<R> w22 = -conjg(cmul(w00, w11) - cmul(w01, w10));
    Link<R> u;  // undo the column reversal
    u.m[0][0] = w02;
    u.m[0][1] = w01;
    u.m[0][2] = w00;
    u.m[1][0] = w12;
    u.m[1][1] = w11;
    u.m[1][2] = w10;
    u.m[2][0] = w22;
    u.m[2][1] = w21;
    u.m[2][2] = w20;
    return u;
}

template <int kRecon, typename R>
__device__ __forceinline__ void reconstruct_row2(Link<R> &u)
{
    if (kRecon == 12) {
        u.m[2][0] = conjg(cmul(u.m[0][1], u.m[1][2]) - cmul(u.m[0][2], u.m[1][1]));
        u.m[2][1] = conjg(cmul(u.m[0][2], u.m[1][0]) - cmul(u.m[0][0], u.m[1][2]));
        u.m[2][2] = conjg(cmul(u.m[0][0], u.m[1][1]) - cmul(u.m[0][1], u.m[1][0]));
    }
}

template <int kRecon>
struct GF64 {
    using R = double;
    static constexpr int kRecon_ = kRecon;
    static constexpr int kPlanes = kRecon / 2;  // double2 (one complex, or two reals of recon-8) per plane
    static constexpr size_t kBytesPerLink = kRecon * 8;
    static constexpr double kTmax = 1e150;      // recon-8 clamp of tan(arg/2)
    struct Raw {
        double2 d[kPlanes];
    };
    __device__ __forceinline__ static Raw fetch(const GaugeView &g, int block, int i)
    {
        Raw r;
        const double2 *p = static_cast<const double2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
        for (int k = 0; k < kPlanes; ++k) r.d[k] = __ldg(p + (size_t)k * g.stride);
        return r;
    }
    __device__ __forceinline__ static Link<R> decode(const Raw &r)
    {
        if constexpr (kRecon == 8) {
            const double p[8] = {r.d[0].x, r.d[0].y, r.d[1].x, r.d[1].y, r.d[2].x, r.d[2].y, r.d[3].x, r.d[3].y};
            return recon8_decode<double>(p);
        } else {
            Link<R> u;
#pragma unroll
            for (int k = 0; k < kPlanes; ++k) u.m[k / 3][k % 3] = mk(r.d[k].x, r.d[k].y);
            reconstruct_row2<kRecon>(u);
            return u;
        }
    }
    __device__ __forceinline__ static Link<R> load(const GaugeView &g, int block, int i) { return decode(fetch(g, block, i)); }
    __device__ __forceinline__ static void store(const GaugeView &g, int block, int i, const Link<R> &u)
    {
        double2 *p = static_cast<double2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
        if constexpr (kRecon == 8) {
            double q[8];
            recon8_encode<double>(u, q, kTmax);
#pragma unroll
            for (int k = 0; k < 4; ++k) p[(size_t)k * g.stride] = make_double2(q[2 * k], q[2 * k + 1]);
        } else {
#pragma unroll
            for (int k = 0; k < kPlanes; ++k)
                p[(size_t)k * g.stride] = make_double2(u.m[k / 3][k % 3].re, u.m[k / 3][k % 3].im);
        }
    }
    __device__ __forceinline__ static void store64(const GaugeView &g, int block, int i, const Link<double> &u)
    {
        store(g, block, i, u);
    }
};

template <int kRecon>
struct GF32 {
    using R = float;
    static constexpr int kRecon_ = kRecon;
    // recon-18: nine float2 planes; recon-12: three float4 planes; recon-8: two float4 planes
    static constexpr int kPlanes = kRecon == 18 ? 9 : kRecon == 12 ? 3 : 2;
    static constexpr size_t kBytesPerLink = kRecon * 4;
    static constexpr float kTmax = 1e18f;  // recon-8 clamp of tan(arg/2) (t^2 stays finite)
    // recon-18: nine float2; recon-12 / recon-8: float4 planes kept as float2 pairs
    struct Raw {
        float2 d[kRecon / 2];
    };
    __device__ __forceinline__ static Raw fetch(const GaugeView &g, int block, int i)
    {
        Raw r;
        if (kRecon == 18) {
            const float2 *p = static_cast<const float2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 9; ++k) r.d[k] = __ldg(p + (size_t)k * g.stride);
        } else {
            const float4 *p = static_cast<const float4 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < kPlanes; ++k) {
                const float4 d = __ldg(p + (size_t)k * g.stride);
                r.d[2 * k] = make_float2(d.x, d.y);
                r.d[2 * k + 1] = make_float2(d.z, d.w);
            }
        }
        return r;
    }
    __device__ __forceinline__ static Link<R> decode(const Raw &r)
    {
        if constexpr (kRecon == 8) {
            const float p[8] = {r.d[0].x, r.d[0].y, r.d[1].x, r.d[1].y, r.d[2].x, r.d[2].y, r.d[3].x, r.d[3].y};
            return recon8_decode<float>(p);
        } else {
            Link<R> u;
#pragma unroll
            for (int k = 0; k < kRecon / 2; ++k) u.m[k / 3][k % 3] = mk(r.d[k].x, r.d[k].y);
            reconstruct_row2<kRecon>(u);
            return u;
        }
    }
    __device__ __forceinline__ static Link<R> load(const GaugeView &g, int block, int i) { return decode(fetch(g, block, i)); }
    __device__ __forceinline__ static void store(const GaugeView &g, int block, int i, const Link<R> &u)
    {
        if (kRecon == 18) {
            float2 *p = static_cast<float2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 9; ++k) p[(size_t)k * g.stride] = make_float2(u.m[k / 3][k % 3].re, u.m[k / 3][k % 3].im);
        } else if (kRecon == 12) {
            float4 *p = static_cast<float4 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const cx<R> a = u.m[(2 * k) / 3][(2 * k) % 3], b = u.m[(2 * k + 1) / 3][(2 * k + 1) % 3];
                p[(size_t)k * g.stride] = make_float4(a.re, a.im, b.re, b.im);
            }
        } else {
            float4 *p = static_cast<float4 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
            float q[8];
            recon8_encode<float>(u, q, kTmax);
            p[0] = make_float4(q[0], q[1], q[2], q[3]);
            p[(size_t)g.stride] = make_float4(q[4], q[5], q[6], q[7]);
        }
    }
    // FP64 source: the recon-8 parameters are computed in FP64 and rounded once
    __device__ __forceinline__ static void store64(const GaugeView &g, int block, int i, const Link<double> &u)
    {
        if constexpr (kRecon == 8) {
            double q[8];
            recon8_encode<double>(u, q, (double)kTmax);
            float4 *p = static_cast<float4 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
            p[0] = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
            p[(size_t)g.stride] = make_float4((float)q[4], (float)q[5], (float)q[6], (float)q[7]);
        } else {
            Link<R> v;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) v.m[a][b] = mk((float)u.m[a][b].re, (float)u.m[a][b].im);
            store(g, block, i, v);
        }
    }
};

// Double-float links: one float4 plane (hi.re, hi.im, lo.re, lo.im) per
// stored complex entry (9 for recon-18, 6 for recon-12).
template <int kRecon>
struct GDF64 {
    using R = df;
    static constexpr int kRecon_ = kRecon;
    static constexpr int kPlanes = kRecon / 2;
    static constexpr size_t kBytesPerLink = kRecon * 8;
    struct Raw {
        float4 d[kPlanes];
    };
    __device__ __forceinline__ static Raw fetch(const GaugeView &g, int block, int i)
    {
        Raw r;
        const float4 *p = static_cast<const float4 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
        for (int k = 0; k < kPlanes; ++k) r.d[k] = __ldg(p + (size_t)k * g.stride);
        return r;
    }
    __device__ __forceinline__ static Link<R> decode(const Raw &r)
    {
        Link<R> u;
#pragma unroll
        for (int k = 0; k < kPlanes; ++k) u.m[k / 3][k % 3] = cx<R>{df(r.d[k].x, r.d[k].z), df(r.d[k].y, r.d[k].w)};
        reconstruct_row2<kRecon>(u);
        return u;
    }
    __device__ __forceinline__ static Link<R> load(const GaugeView &g, int block, int i) { return decode(fetch(g, block, i)); }
    __device__ __forceinline__ static void store(const GaugeView &g, int block, int i, const Link<R> &u)
    {
        float4 *p = static_cast<float4 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
        for (int k = 0; k < kPlanes; ++k) {
            const cx<R> a = u.m[k / 3][k % 3];
            p[(size_t)k * g.stride] = make_float4(a.re.hi, a.im.hi, a.re.lo, a.im.lo);
        }
    }
    __device__ __forceinline__ static void store64(const GaugeView &g, int block, int i, const Link<double> &u)
    {
        Link<R> v;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) v.m[a][b] = cx<R>{df(u.m[a][b].re), df(u.m[a][b].im)};
        store(g, block, i, v);
    }
};

// 16-bit links (FP16 or BF16), unscaled (|U_ab| <= 1).  recon-18: nine
// 4-byte planes (one complex); recon-12: three 8-byte planes (two complex).
template <typename H, int kRecon>
struct G16 {
    using R = float;
    static constexpr int kRecon_ = kRecon;
    static constexpr int kPlanes = kRecon == 18 ? 9 : kRecon == 12 ? 3 : 1;
    static constexpr size_t kBytesPerLink = kRecon * 2;
    // recon-8 clamp of tan(arg/2): inside the FP16 range (BF16 has the FP32 range)
    static constexpr double kTmax = std::is_same<H, __half>::value ? 32768.0 : 1e18;
    // one 32-bit word (two 16-bit reals) per complex entry / recon-8 pair
    struct Raw {
        uint32_t w[kRecon / 2];
    };
    __device__ __forceinline__ static Raw fetch(const GaugeView &g, int block, int i)
    {
        Raw r;
        if (kRecon == 18) {
            const uint32_t *p = static_cast<const uint32_t *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 9; ++k) r.w[k] = __ldg(p + (size_t)k * g.stride);
        } else if (kRecon == 12) {
            const uint2 *p = static_cast<const uint2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const uint2 w = __ldg(p + (size_t)k * g.stride);
                r.w[2 * k] = w.x;
                r.w[2 * k + 1] = w.y;
            }
        } else {
            const uint4 w = __ldg(static_cast<const uint4 *>(g.data) + (size_t)block * g.stride + i);
            r.w[0] = w.x;
            r.w[1] = w.y;
            r.w[2] = w.z;
            r.w[3] = w.w;
        }
        return r;
    }
    __device__ __forceinline__ static Link<R> decode(const Raw &r)
    {
        if constexpr (kRecon == 8) {
            float p[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = Half16<H>::to2(r.w[k]);
                p[2 * k] = f.x;
                p[2 * k + 1] = f.y;
            }
            return recon8_decode<float>(p);
        } else {
            Link<R> u;
#pragma unroll
            for (int k = 0; k < kRecon / 2; ++k) {
                const float2 f = Half16<H>::to2(r.w[k]);
                u.m[k / 3][k % 3] = mk(f.x, f.y);
            }
            reconstruct_row2<kRecon>(u);
            return u;
        }
    }
    __device__ __forceinline__ static Link<R> load(const GaugeView &g, int block, int i) { return decode(fetch(g, block, i)); }
    __device__ __forceinline__ static void store_params(const GaugeView &g, int block, int i, const float q[8])
    {
        uint4 *p = static_cast<uint4 *>(g.data) + (size_t)block * g.stride + i;
        *p = make_uint4(Half16<H>::from2(q[0], q[1]), Half16<H>::from2(q[2], q[3]), Half16<H>::from2(q[4], q[5]),
                        Half16<H>::from2(q[6], q[7]));
    }
    __device__ __forceinline__ static void store(const GaugeView &g, int block, int i, const Link<R> &u)
    {
        if (kRecon == 18) {
            uint32_t *p = static_cast<uint32_t *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 9; ++k) p[(size_t)k * g.stride] = Half16<H>::from2(u.m[k / 3][k % 3].re, u.m[k / 3][k % 3].im);
        } else if (kRecon == 12) {
            uint2 *p = static_cast<uint2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const cx<R> a = u.m[(2 * k) / 3][(2 * k) % 3], b = u.m[(2 * k + 1) / 3][(2 * k + 1) % 3];
                p[(size_t)k * g.stride] = make_uint2(Half16<H>::from2(a.re, a.im), Half16<H>::from2(b.re, b.im));
            }
        } else {
            float q[8];
            recon8_encode<float>(u, q, (float)kTmax);
            store_params(g, block, i, q);
        }
    }
    // FP64 source: the recon-8 parameters are computed in FP64 and rounded once to FP32, then to 16 bits
    __device__ __forceinline__ static void store64(const GaugeView &g, int block, int i, const Link<double> &u)
    {
        if constexpr (kRecon == 8) {
            double q[8];
            recon8_encode<double>(u, q, kTmax);
            float f[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) f[k] = (float)q[k];
            store_params(g, block, i, f);
        } else {
            Link<R> v;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) v.m[a][b] = mk((float)u.m[a][b].re, (float)u.m[a][b].im);
            store(g, block, i, v);
        }
    }
};

// Bytes of one plane element of each format (host side, for allocation).
size_t spinor_plane_elem_bytes(int prec);
int spinor_planes(int prec);
size_t gauge_plane_elem_bytes(int prec, int recon);
int gauge_planes(int prec, int recon);

// ------------------------------------------------------------------ geometry

// Division by a fixed divisor d through one 64-bit multiply: q = (n m) >> 32
// with m = ceil(2^32 / d).  Exact whenever n * d < 2^32 (checked when the
// lattice is created).
struct FastDiv {
    uint64_t m;
    uint32_t d;
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return (uint32_t)(((uint64_t)n * m) >> 32); }
};
inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d;
    f.m = ((1ull << 32) + d - 1) / d;
    return f;
}

struct Geom {
    int L[4];       // Lx, Ly, Lz, Lt (all even)
    int Lxh;        // Lx / 2
    int h;          // V / 2 sites per parity
    int sy, sz, st; // half-index strides of y, z, t: Lxh, Lxh Ly, Lxh Ly Lz
    FastDiv dx, dy, dz;
    double tbc;     // factor of the hop that wraps in t
};

// tbc < 0 as a test of its sign bit: an integer instruction, where the
// double comparison would take the FP64 pipe in the FP32 and 16-bit kernels.
__device__ __forceinline__ bool antiperiodic(const Geom &g) { return __double_as_longlong(g.tbc) < 0; }

// Coordinates of half-site i of parity p.
struct SiteCoords {
    int x, y, z, t, xh;
};
__device__ __forceinline__ SiteCoords site_coords(const Geom &g, int i, int p)
{
    SiteCoords c;
    uint32_t r = g.dx.div((uint32_t)i);
    c.xh = i - (int)r * g.Lxh;
    uint32_t r2 = g.dy.div(r);
    c.y = (int)r - (int)r2 * g.L[1];
    uint32_t r3 = g.dz.div(r2);
    c.z = (int)r2 - (int)r3 * g.L[2];
    c.t = (int)r3;
    c.x = 2 * c.xh + ((c.y + c.z + c.t + p) & 1);
    return c;
}

// ------------------------------------------------------------------ reductions

// Deterministic block reduction of NV doubles: warp shuffles, then a fixed
// tree over warps.  The returned values are valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *smem /* NV * 32 */)
{
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) smem[k * 32 + warp] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < nw ? smem[k * 32 + lane] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            v[k] = s;
        }
    }
}

// Scratch of a grid-wide reduction in up to two levels: one partial per
// block; blocks form groups of red_group_size(gridDim.x, P) consecutive
// blocks (P reduced quantities), and the last block of a group to finish
// sums the group's partials in block order; with several groups, the last
// group to finish then sums the group sums in group order.  The result does
// not depend on scheduling, and no block sums more than about 2048 values
// (or sqrt(gridDim.x) per quantity): a single last block summing every
// partial took longer than the kernel itself for batched fields.
struct Reduction {
    double *partials;   // >= red_partials_needed(NV * nrhs, gridDim.x) doubles
    unsigned *counter;  // 1 + groups tickets, zero before the launch; reset by the finishing blocks
    size_t cap;         // capacity of partials in doubles (checked on the host before each launch)
};

// Blocks per group for P reduced quantities: a power of two >= 64 and
// >= 2048 / P (so one level suffices for small grids), with at most as many
// groups as blocks per group.  Not smaller for more blocks or fewer
// quantities.
__host__ __device__ inline unsigned red_group_size(unsigned blocks, unsigned P)
{
    unsigned g = 64;
    while (g * P < 2048) g <<= 1;
    while ((blocks + g - 1) / g > g) g <<= 1;
    return g;
}
// Doubles of partials for `quantities` reduced values (values x rhs) over
// at most `blocks` blocks: the block partials, then the group sums (fewer
// than the group size, which does not decrease with the block count, so
// the bound holds for every smaller grid too).
inline size_t red_partials_needed(size_t quantities, size_t blocks)
{
    return quantities * (blocks + red_group_size((unsigned)blocks, (unsigned)quantities));
}

// Host check: a reducing launch of `blocks` blocks with NV values for 2^L
// right-hand sides fits the partials buffer.
inline bool reduction_fits(const Reduction &r, int nv, int rhs_log2, size_t blocks)
{
    return blocks < (1u << 31) && red_partials_needed((size_t)nv << rhs_log2, blocks) <= r.cap;
}

// Device-resident CG state for nrhs right-hand sides solved together.
// Kernels of an iteration read the global `status` and return at once when
// it is not RUNNING, so the host may enqueue iterations ahead without reading
// anything back.  Each right-hand side keeps its own scalars: a solved one
// gets alpha = beta = 0 and rides along unchanged.
enum CgStatus : int {
    CG_RUNNING = 0,
    CG_CONVERGED = 1,   // (per rhs) iterated residual below the target
    CG_RELIABLE = 2,    // (global) an FP64 true residual is due
    CG_BREAKDOWN = 3,   // <p, A p> <= 0 or non-finite values
    CG_MAXITER = 4,     // (global)
    CG_DONE = 5,        // true residual below the target
    CG_VERIFY = 6,      // (global) an inner-precision estimate of the true residual met a target: check in FP64
};

constexpr int kMaxRhs = 32;

struct CgRhs {
    double rr;        // |r|^2 of the current iterate
    double rr_prev;   // |r|^2 before the last update (beta after a reliable update)
    double pAp;       // |Mhat p|^2 of this iteration
    double alpha, beta;
    double rr_stop;   // tol^2 |rhs|^2
    double rr_max;    // largest |r|^2 since the last reliable update
    double rr_true;   // |rhs - A x|^2 of the last true-residual computation
    double b2;        // |rhs|^2
    double tol2;      // this rhs's target relative residual, squared
    int status;       // RUNNING, DONE or BREAKDOWN
    int iter_done;    // iteration at which it was solved
};

struct CgState {
    CgRhs r[kMaxRhs];
    int nrhs;
    double tol2;      // tol^2
    double delta2;    // reliable_delta^2 (0: true residual only at convergence)
    int iter, maxiter;
    int status;       // global
    int reliable_updates;
    int trips, trip_limit;  // device-driven loop: body executions and their cap
};

// What the last block does with a finished reduction.
enum FinalizeKind : int {
    FIN_STORE = 0,      // out[k * nrhs + r] = totals
    FIN_CG_ALPHA = 1,   // pAp = total; alpha = rr / pAp (breakdown check)
    FIN_CG_RR = 2,      // rr_new = total; beta, convergence, reliable trigger
    FIN_CG_TRUE = 3,    // true residual after a reliable update
    FIN_CG_INIT = 4,    // |rhs|^2 at the start of CG
    FIN_CG_TRUE_EST = 5,// true residual estimated in the inner precision (Mhat^dag of the FP64 defect)
};

// tot[r] = the reduced value of right-hand side r (first value only).
__device__ __forceinline__ void cg_finalize_rhs(FinalizeKind kind, const double *tot, CgState *st)
{
    const int n = st->nrhs;
    if (kind == FIN_CG_INIT) {
        bool all_done = true, bad = false;
        for (int k = 0; k < n; ++k) {
            CgRhs &q = st->r[k];
            const double b2 = tot[k];
            q.rr = q.rr_prev = q.rr_max = q.rr_true = q.b2 = b2;
            q.rr_stop = q.tol2 * b2;
            q.alpha = q.beta = q.pAp = 0.0;
            q.iter_done = 0;
            q.status = b2 == 0.0 ? CG_DONE : CG_RUNNING;
            all_done = all_done && q.status == CG_DONE;
            bad = bad || !isfinite(b2);
        }
        st->iter = 0;
        st->reliable_updates = 0;
        st->status = bad ? CG_BREAKDOWN : all_done ? CG_DONE : CG_RUNNING;
    } else if (kind == FIN_CG_ALPHA) {
        for (int k = 0; k < n; ++k) {
            CgRhs &q = st->r[k];
            q.pAp = tot[k];
            if (q.status == CG_DONE) {
                q.alpha = 0.0;
            } else if (!(tot[k] > 0.0) || !isfinite(tot[k])) {
                q.alpha = 0.0;
                q.status = CG_BREAKDOWN;
                st->status = CG_BREAKDOWN;
            } else {
                q.alpha = q.rr / tot[k];
            }
        }
    } else if (kind == FIN_CG_RR) {
        // A true-residual update runs when every running system is ready --
        // its residual fell by the reliable-update factor delta since the last
        // update, or it meets its target -- or when some system's residual
        // fell by delta^2 (so one slow system cannot hold the others back).
        // A batch of similar systems thus pays about the updates of one
        // solve, and one final check rather than one per system.
        st->iter += 1;
        bool all_ready = true, urgent = false, bad = false;
        const double d2 = st->delta2;
        for (int k = 0; k < n; ++k) {
            CgRhs &q = st->r[k];
            if (q.status == CG_DONE) {
                q.beta = 0.0;
                continue;
            }
            const double rr_new = tot[k];
            q.rr_prev = q.rr;
            q.beta = rr_new / q.rr;
            q.rr = rr_new;
            if (!isfinite(rr_new)) bad = true;
            const bool dropped = d2 > 0.0 && rr_new < d2 * q.rr_max;
            all_ready = all_ready && (dropped || rr_new <= q.rr_stop);
            urgent = urgent || (d2 > 0.0 && rr_new < d2 * d2 * q.rr_max);
            if (rr_new > q.rr_max) q.rr_max = rr_new;
        }
        if (bad)
            st->status = CG_BREAKDOWN;
        else if (all_ready || urgent)
            st->status = CG_RELIABLE;
        else if (st->iter >= st->maxiter)
            st->status = CG_MAXITER;
    } else if (kind == FIN_CG_TRUE_EST) {
        // The FP64 defect rho = rhs0 - Mhat x, mapped by Mhat^dag in a lower
        // precision: a system whose estimate meets its target is checked in
        // FP64 next (CG_VERIFY); the others continue from the estimate.
        st->reliable_updates += 1;
        bool verify = false, bad = false;
        for (int k = 0; k < n; ++k) {
            CgRhs &q = st->r[k];
            if (q.status == CG_DONE) {
                q.beta = 0.0;
                continue;
            }
            const double rt = tot[k];
            q.rr_true = rt;
            if (!isfinite(rt)) {
                bad = true;
            } else if (rt <= q.rr_stop) {
                verify = true;
            } else {
                q.beta = rt / q.rr_prev;
                q.rr = rt;
                q.rr_max = rt;
            }
        }
        st->status = bad ? CG_BREAKDOWN : verify ? CG_VERIFY : (st->iter >= st->maxiter ? CG_MAXITER : CG_RUNNING);
    } else if (kind == FIN_CG_TRUE) {
        if (st->status != CG_VERIFY) st->reliable_updates += 1;  // (a verification completes its update)
        bool all_done = true, bad = false;
        for (int k = 0; k < n; ++k) {
            CgRhs &q = st->r[k];
            if (q.status == CG_DONE) {
                q.beta = 0.0;
                continue;
            }
            const double rt = tot[k];
            q.rr_true = rt;
            if (!isfinite(rt)) {
                bad = true;
            } else if (rt <= q.rr_stop) {
                q.status = CG_DONE;
                q.iter_done = st->iter;
                q.beta = 0.0;
            } else {
                q.beta = rt / q.rr_prev;
                q.rr = rt;
                q.rr_max = rt;
            }
            all_done = all_done && q.status == CG_DONE;
        }
        st->status = bad ? CG_BREAKDOWN
                         : all_done ? CG_DONE : (st->iter >= st->maxiter ? CG_MAXITER : CG_RUNNING);
    }
}

// Grid-wide reduction segmented by right-hand side: element e of a batched
// field belongs to rhs e & (nrhs - 1) (nrhs a power of two <= 32, the rhs
// index fastest), so in a warp the lanes of one rhs are lane & (nrhs - 1).
// NV values per element; the last block sums the per-block partials of each
// (value, rhs) in block order and finalises.  All threads must call it;
// blockDim.x must be a multiple of 32 and at most 256.
// Sums of P rows of `count` doubles (row q at src + q * stride), by every
// thread of the block: T = blockDim / P threads per row (at least one; P and
// blockDim powers of two), each taking every T-th element from its offset
// with four accumulators (loads in flight), then the T sums of a row added
// by a fixed binary tree into res[q] (shared).  The order is fixed, so the
// sums are reproducible.
__device__ __forceinline__ void block_row_sums(const double *src, size_t stride, int P, unsigned count,
                                               double *res, double *scratch /* blockDim.x */)
{
    const int T = (int)blockDim.x >= P ? (int)blockDim.x / P : 1;
    const int rows_per_pass = (int)blockDim.x / T;
    for (int q0 = 0; q0 < P; q0 += rows_per_pass) {
        const int q = q0 + (int)threadIdx.x / T, j = (int)threadIdx.x % T;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        if (q < P) {
            const double *row = src + (size_t)q * stride;
            unsigned b = j;
            for (; b + 3u * T < count; b += 4u * T) {
                a0 += __ldcg(row + b);
                a1 += __ldcg(row + b + T);
                a2 += __ldcg(row + b + 2u * T);
                a3 += __ldcg(row + b + 3u * T);
            }
            for (; b < count; b += T) a0 += __ldcg(row + b);
        }
        scratch[threadIdx.x] = (a0 + a1) + (a2 + a3);
        __syncthreads();
        for (int off = T >> 1; off > 0; off >>= 1) {
            if (j < off) scratch[threadIdx.x] += scratch[threadIdx.x + off];
            __syncthreads();
        }
        if (j == 0 && q < P) res[q] = scratch[threadIdx.x];
        __syncthreads();
    }
}

// (grid_reduce_rhs after the sums within each warp: lane r < nrhs holds
// the warp's sum of rhs r)
template <int NV>
__device__ __forceinline__ void grid_reduce_rhs_warp_summed(const double (&v)[NV], int rhs_log2, const Reduction &red,
                                                            FinalizeKind kind, CgState *st, double *out)
{
    __shared__ double sw[NV][8][kMaxRhs];  // [value][warp][rhs]; blocks of <= 256 threads
    __shared__ double tot[NV * kMaxRhs];
    __shared__ double scratch[256];
    __shared__ bool is_last;
    const int n = 1 << rhs_log2, P = NV * n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned nb = gridDim.x, G = red_group_size(nb, P), ng = (nb + G - 1) / G, grp = blockIdx.x / G;
    const unsigned gsize = nb - grp * G < G ? nb - grp * G : G;
    if (lane < n)
#pragma unroll
        for (int k = 0; k < NV; ++k) sw[k][warp][lane] = v[k];
    __syncthreads();
    if ((int)threadIdx.x < P) {
        const int k = threadIdx.x / n, r = threadIdx.x % n;
        double b = 0.0;
        for (int w = 0; w < nw; ++w) b += sw[k][w][r];
        red.partials[((size_t)k * n + r) * nb + blockIdx.x] = b;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(red.counter + 1 + grp, 1u) == gsize - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // the last block of the group: the group's partials in block order
    block_row_sums(red.partials + (size_t)grp * G, nb, P, gsize, tot, scratch);
    if (ng > 1) {
        double *gsum = red.partials + (size_t)P * nb;
        if ((int)threadIdx.x < P) {
            gsum[(size_t)threadIdx.x * ng + grp] = tot[threadIdx.x];
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            red.counter[1 + grp] = 0u;
            is_last = atomicAdd(red.counter, 1u) == ng - 1;
        }
        __syncthreads();
        if (!is_last) return;
        __threadfence();
        // the last group: the group sums in group order
        block_row_sums(gsum, ng, P, ng, tot, scratch);
    }
    if (threadIdx.x == 0) {
        red.counter[1] = 0u;  // (one group: its ticket; otherwise already reset)
        if (kind == FIN_STORE) {
            for (int q = 0; q < NV * n; ++q) out[q] = tot[q];
        } else {
            cg_finalize_rhs(kind, tot, st);
        }
        *red.counter = 0u;
    }
}

template <int NV>
__device__ __forceinline__ void grid_reduce_rhs(double (&v)[NV], int rhs_log2, const Reduction &red,
                                                FinalizeKind kind, CgState *st, double *out)
{
    const int n = 1 << rhs_log2;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int off = 16; off >= n; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    grid_reduce_rhs_warp_summed<NV>(v, rhs_log2, red, kind, st, out);
}

// The same for FP32 values (the FP32 and 16-bit kernels' inner-solver
// norms): the sums within a warp are taken in float, so a warp issues one
// float-to-double conversion instead of five FP64 additions (FP64
// instructions hold the FP64 pipe 64 cycles per warp); the block and grid
// sums stay in double and in a fixed order.
template <int NV>
__device__ __forceinline__ void grid_reduce_rhs(float (&vf)[NV], int rhs_log2, const Reduction &red,
                                                FinalizeKind kind, CgState *st, double *out)
{
    const int n = 1 << rhs_log2;
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        for (int off = 16; off >= n; off >>= 1) vf[k] += __shfl_xor_sync(0xffffffffu, vf[k], off);
        v[k] = (double)vf[k];
    }
    grid_reduce_rhs_warp_summed<NV>(v, rhs_log2, red, kind, st, out);
}

// ------------------------------------------------------------------ launch API

// Epilogue of the hopping kernel: out = cy .* y + cd .* (D psi), with one
// complex coefficient per chirality (upper spins 0,1 / lower spins 2,3).
// This covers A y - kappa^2 D psi, A^-1 D psi, y + kappa D psi, and their
// adjoints, for A = 1 + i a gamma_5.
enum EpiMode : int {
    EPI_PLAIN = 0,     // out = D psi
    EPI_REAL_D = 1,    // out = cd.re * D psi                     (real scale)
    EPI_REAL_YD = 2,   // out = cy.re * y + cd.re * D psi         (Wilson)
    EPI_CPLX_D = 3,    // out = cd[chi] * D psi                   (twisted)
    EPI_CPLX_YD = 4,   // out = cy[chi] * y + cd[chi] * D psi     (twisted)
};

// Arguments of one hopping-kernel launch.  in/out/y are indexed by the
// output parity p (in[p] holds the sites of parity 1-p).  With both = 1 the
// launch covers both output parities (the full-lattice operator).
struct DslashLaunch {
    Geom g;
    int out_parity;
    int both;
    int rhs_log2;       // batched fields: element = site * 2^rhs_log2 + rhs
    int tpb;            // threads per block (FP32/16-bit kernels; 0: default)
    int split;          // threads per output site: 1 (0), or 8 (FP64 reconstruct-18, one rhs)
    int tmap;           // 0, or blocks per time slice: blocks run in t-major order (batched fields)
    int dagger;
    GaugeView U;
    SpinorView in[2], out[2], y[2];
    double cy[2][2], cd[2][2];  // [chirality][re, im]
    float cyf[2][2], cdf[2][2]; // the same rounded to float (FP32 and 16-bit kernels)
    const double *coef;         // if set: cy, cd read from this device table (8 doubles) instead
    const float *coef_f;        // its float image (same layout), read by the FP32 and 16-bit kernels
    int coef_stride;            // entries between the tables of consecutive rhs (0: one table for all)
    EpiMode epi;
    // optional fused |out|^2 reduction
    bool reduce;
    Reduction red;
    FinalizeKind fin;
    CgState *state;     // also: early exit when state->status != run_status (if check_status)
    double *red_out;
    bool check_status;
    int run_status;     // the status the launch runs under (CG_RUNNING, or CG_VERIFY for a check)
};

cudaError_t launch_dslash(int prec, int recon, const DslashLaunch &a, cudaStream_t s);

// number of blocks / threads used by site kernels (for scratch sizing)
constexpr int kThreads = 128;
inline int site_blocks(int n) { return (n + kThreads - 1) / kThreads; }

}  // namespace qcd
