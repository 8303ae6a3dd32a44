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

// Gauge storage formats: kRecon = 18 (full matrix) or 12 (rows 0 and 1;
// row 2 = conj(row0 x row1), valid for SU(3)).
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
    static constexpr int kPlanes = kRecon / 2;  // double2 (one complex) per plane
    static constexpr size_t kBytesPerLink = kRecon * 8;
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
        Link<R> u;
#pragma unroll
        for (int k = 0; k < kPlanes; ++k) u.m[k / 3][k % 3] = mk(r.d[k].x, r.d[k].y);
        reconstruct_row2<kRecon>(u);
        return u;
    }
    __device__ __forceinline__ static Link<R> load(const GaugeView &g, int block, int i)
    {
        Link<R> u;
        const double2 *p = static_cast<const double2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
        for (int k = 0; k < kPlanes; ++k) {
            double2 d = __ldg(p + (size_t)k * g.stride);
            u.m[k / 3][k % 3] = mk(d.x, d.y);
        }
        reconstruct_row2<kRecon>(u);
        return u;
    }
    __device__ __forceinline__ static void store(const GaugeView &g, int block, int i, const Link<R> &u)
    {
        double2 *p = static_cast<double2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
        for (int k = 0; k < kPlanes; ++k) p[(size_t)k * g.stride] = make_double2(u.m[k / 3][k % 3].re, u.m[k / 3][k % 3].im);
    }
};

template <int kRecon>
struct GF32 {
    using R = float;
    static constexpr int kRecon_ = kRecon;
    // recon-18: nine float2 planes; recon-12: three float4 planes
    static constexpr int kPlanes = kRecon == 18 ? 9 : 3;
    static constexpr size_t kBytesPerLink = kRecon * 4;
    // recon-18: nine float2; recon-12: three float4 (kept as six float2)
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
            for (int k = 0; k < 3; ++k) {
                const float4 d = __ldg(p + (size_t)k * g.stride);
                r.d[2 * k] = make_float2(d.x, d.y);
                r.d[2 * k + 1] = make_float2(d.z, d.w);
            }
        }
        return r;
    }
    __device__ __forceinline__ static Link<R> decode(const Raw &r)
    {
        Link<R> u;
#pragma unroll
        for (int k = 0; k < kRecon / 2; ++k) u.m[k / 3][k % 3] = mk(r.d[k].x, r.d[k].y);
        reconstruct_row2<kRecon>(u);
        return u;
    }
    __device__ __forceinline__ static Link<R> load(const GaugeView &g, int block, int i)
    {
        Link<R> u;
        if (kRecon == 18) {
            const float2 *p = static_cast<const float2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                float2 d = __ldg(p + (size_t)k * g.stride);
                u.m[k / 3][k % 3] = mk(d.x, d.y);
            }
        } else {
            const float4 *p = static_cast<const float4 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float4 d = __ldg(p + (size_t)k * g.stride);
                u.m[(2 * k) / 3][(2 * k) % 3] = mk(d.x, d.y);
                u.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(d.z, d.w);
            }
            reconstruct_row2<12>(u);
        }
        return u;
    }
    __device__ __forceinline__ static void store(const GaugeView &g, int block, int i, const Link<R> &u)
    {
        if (kRecon == 18) {
            float2 *p = static_cast<float2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 9; ++k) p[(size_t)k * g.stride] = make_float2(u.m[k / 3][k % 3].re, u.m[k / 3][k % 3].im);
        } else {
            float4 *p = static_cast<float4 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const cx<R> a = u.m[(2 * k) / 3][(2 * k) % 3], b = u.m[(2 * k + 1) / 3][(2 * k + 1) % 3];
                p[(size_t)k * g.stride] = make_float4(a.re, a.im, b.re, b.im);
            }
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
};

// 16-bit links (FP16 or BF16), unscaled (|U_ab| <= 1).  recon-18: nine
// 4-byte planes (one complex); recon-12: three 8-byte planes (two complex).
template <typename H, int kRecon>
struct G16 {
    using R = float;
    static constexpr int kRecon_ = kRecon;
    static constexpr int kPlanes = kRecon == 18 ? 9 : 3;
    static constexpr size_t kBytesPerLink = kRecon * 2;
    // one 32-bit word (two 16-bit reals) per complex entry
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
        } else {
            const uint2 *p = static_cast<const uint2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const uint2 w = __ldg(p + (size_t)k * g.stride);
                r.w[2 * k] = w.x;
                r.w[2 * k + 1] = w.y;
            }
        }
        return r;
    }
    __device__ __forceinline__ static Link<R> decode(const Raw &r)
    {
        Link<R> u;
#pragma unroll
        for (int k = 0; k < kRecon / 2; ++k) {
            const float2 f = Half16<H>::to2(r.w[k]);
            u.m[k / 3][k % 3] = mk(f.x, f.y);
        }
        reconstruct_row2<kRecon>(u);
        return u;
    }
    __device__ __forceinline__ static Link<R> load(const GaugeView &g, int block, int i)
    {
        Link<R> u;
        if (kRecon == 18) {
            const uint32_t *p = static_cast<const uint32_t *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                float2 f = Half16<H>::to2(__ldg(p + (size_t)k * g.stride));
                u.m[k / 3][k % 3] = mk(f.x, f.y);
            }
        } else {
            const uint2 *p = static_cast<const uint2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                uint2 w = __ldg(p + (size_t)k * g.stride);
                float2 a = Half16<H>::to2(w.x), b = Half16<H>::to2(w.y);
                u.m[(2 * k) / 3][(2 * k) % 3] = mk(a.x, a.y);
                u.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(b.x, b.y);
            }
            reconstruct_row2<12>(u);
        }
        return u;
    }
    __device__ __forceinline__ static void store(const GaugeView &g, int block, int i, const Link<R> &u)
    {
        if (kRecon == 18) {
            uint32_t *p = static_cast<uint32_t *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 9; ++k) p[(size_t)k * g.stride] = Half16<H>::from2(u.m[k / 3][k % 3].re, u.m[k / 3][k % 3].im);
        } else {
            uint2 *p = static_cast<uint2 *>(g.data) + (size_t)block * kPlanes * g.stride + i;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const cx<R> a = u.m[(2 * k) / 3][(2 * k) % 3], b = u.m[(2 * k + 1) / 3][(2 * k + 1) % 3];
                p[(size_t)k * g.stride] = make_uint2(Half16<H>::from2(a.re, a.im), Half16<H>::from2(b.re, b.im));
            }
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

// Scratch of a grid-wide reduction: one partial per block and a ticket
// counter; the last block to finish sums the partials in block order, so
// the result does not depend on scheduling.
struct Reduction {
    double *partials;   // >= gridDim.x * NV doubles
    unsigned *counter;  // zero before the launch; reset to zero by the last block
};

// Device-resident CG state.  Kernels of an iteration read `status` and
// return at once when it is not RUNNING, so the host may enqueue several
// iterations ahead without reading anything back.
enum CgStatus : int {
    CG_RUNNING = 0,
    CG_CONVERGED = 1,   // iterated residual below the target
    CG_RELIABLE = 2,    // reliable update requested
    CG_BREAKDOWN = 3,   // <p, A p> <= 0 or not finite
    CG_MAXITER = 4,
    CG_DONE = 5,        // true residual below the target: solved
};

struct CgState {
    double rr;        // |r|^2 of the current iterate
    double rr_prev;   // |r|^2 before the last update (for beta after a reliable update)
    double pAp;       // |Mhat p|^2 of this iteration
    double alpha, beta;
    double rr_stop;   // tol^2 |rhs|^2
    double rr_max;    // largest |r|^2 since the last reliable update
    double delta2;    // reliable_delta^2 (0: no reliable updates)
    double rr_true;   // |rhs - A x|^2 from the last true-residual computation
    double tol2;      // tol^2
    double b2;        // |rhs|^2
    int iter, maxiter;
    int status;
    int reliable_updates;
    int trips, trip_limit;  // device-driven loop: body executions and their cap
    unsigned counter[4];
};

// What the last block does with a finished reduction.
enum FinalizeKind : int {
    FIN_STORE = 0,      // out[0..NV) = totals
    FIN_CG_ALPHA = 1,   // pAp = total; alpha = rr / pAp (breakdown check)
    FIN_CG_RR = 2,      // rr_new = total; beta, convergence, reliable trigger
    FIN_CG_TRUE = 3,    // true residual after a reliable update
    FIN_CG_INIT = 4,    // |rhs|^2 at the start of CG
};

template <int NV>
__device__ __forceinline__ void cg_finalize(FinalizeKind kind, const double (&tot)[NV], CgState *st, double *out)
{
    if (kind == FIN_CG_INIT) {
        const double b2 = tot[0];
        st->rr = st->rr_prev = st->rr_max = st->rr_true = b2;
        st->rr_stop = st->tol2 * b2;
        st->b2 = b2;
        st->iter = 0;
        st->reliable_updates = 0;
        st->alpha = st->beta = 0.0;
        st->status = (b2 == 0.0) ? CG_DONE : (isfinite(b2) ? CG_RUNNING : CG_BREAKDOWN);
    } else if (kind == FIN_STORE) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = tot[k];
    } else if (kind == FIN_CG_ALPHA) {
        const double pAp = tot[0];
        st->pAp = pAp;
        if (!(pAp > 0.0) || !isfinite(pAp)) {
            st->status = CG_BREAKDOWN;
            st->alpha = 0.0;
        } else {
            st->alpha = st->rr / pAp;
        }
    } else if (kind == FIN_CG_RR) {
        const double rr_new = tot[0];
        st->iter += 1;
        st->rr_prev = st->rr;
        st->beta = rr_new / st->rr;
        st->rr = rr_new;
        if (!isfinite(rr_new)) {
            st->status = CG_BREAKDOWN;
        } else if (rr_new <= st->rr_stop) {
            st->status = st->delta2 > 0.0 ? CG_RELIABLE : CG_CONVERGED;
        } else if (st->delta2 > 0.0 && rr_new < st->delta2 * st->rr_max) {
            st->status = CG_RELIABLE;
        } else if (st->iter >= st->maxiter) {
            st->status = CG_MAXITER;
        }
        if (rr_new > st->rr_max) st->rr_max = rr_new;
    } else if (kind == FIN_CG_TRUE) {
        // rr_true = |rhs - A x|^2 with x the accumulated solution.
        const double rt = tot[0];
        st->rr_true = rt;
        st->reliable_updates += 1;
        if (!isfinite(rt)) {
            st->status = CG_BREAKDOWN;
        } else if (rt <= st->rr_stop) {
            st->status = CG_DONE;
        } else if (st->iter >= st->maxiter) {
            st->status = CG_MAXITER;
        } else {
            st->beta = rt / st->rr_prev;
            st->rr = rt;
            st->rr_max = rt;
            st->status = CG_RUNNING;
        }
    }
}

// Grid-wide deterministic reduction of NV doubles per thread with the
// last-block pattern.  All threads of the block must call it.
template <int NV>
__device__ __forceinline__ void grid_reduce(double (&v)[NV], const Reduction &red, FinalizeKind kind, CgState *st,
                                            double *out)
{
    __shared__ double smem[NV * 32];
    __shared__ bool is_last;
    block_sum<NV>(v, smem);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) red.partials[(size_t)k * gridDim.x + blockIdx.x] = v[k];
        __threadfence();
        const unsigned ticket = atomicAdd(red.counter, 1u);
        is_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        s[k] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s[k] += __ldcg(red.partials + (size_t)k * gridDim.x + b);
    }
    block_sum<NV>(s, smem);
    if (threadIdx.x == 0) {
        cg_finalize<NV>(kind, s, st, out);
        *red.counter = 0u;
    }
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
    int dagger;
    GaugeView U;
    SpinorView in[2], out[2], y[2];
    double cy[2][2], cd[2][2];  // [chirality][re, im]
    EpiMode epi;
    // optional fused |out|^2 reduction
    bool reduce;
    Reduction red;
    FinalizeKind fin;
    CgState *state;     // also: early exit when state->status != RUNNING (if check_status)
    double *red_out;
    bool check_status;
};

cudaError_t launch_dslash(int prec, int recon, const DslashLaunch &a, cudaStream_t s);

// number of blocks / threads used by site kernels (for scratch sizing)
constexpr int kThreads = 128;
inline int site_blocks(int n) { return (n + kThreads - 1) / kThreads; }

}  // namespace qcd
