// Staggered (Kogut-Susskind) hopping kernel D_KS and the layout kernels of
// staggered fields.
//
// CL2QCD's second Dirac operator (arXiv:1411.5219, Sec. 1 and Sec. 6): on
// one-component colour vectors,
//
//   (D_KS chi)(x) = sum_mu eta_mu(x) [ U_mu(x) chi(x+mu) - U_mu(x-mu)^dagger chi(x-mu) ],
//   eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z),
//
// with the factor t_bc on hops that wrap in time.  The paper counts 570 flop
// and 1584 bytes per site (no neighbour reuse); here, with every link and
// input vector read once, the compulsory traffic is 8 links + 2 vectors.
// Like the Wilson hopping term it connects even and odd sites only.  One
// thread computes one output site; links use the same per-(parity, mu)
// block layout and storage formats as the Wilson kernels.
#include "qcd_ops.h"

namespace qcd {
namespace {

template <typename R>
struct Colour {
    cx<R> c[3];
};

// Staggered field formats: three planes, one complex per plane.
struct KS64 {
    using R = double;
    static constexpr bool kScaled = false;
    __device__ __forceinline__ static Colour<R> load(const SpinorView &v, int i, R &w)
    {
        Colour<R> r;
        const double2 *p = static_cast<const double2 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double2 d = __ldg(p + (size_t)k * v.stride);
            r.c[k] = mk(d.x, d.y);
        }
        w = 1.0;
        return r;
    }
    __device__ __forceinline__ static void store(const SpinorView &v, int i, const Colour<R> &r)
    {
        double2 *p = static_cast<double2 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) p[(size_t)k * v.stride] = make_double2(r.c[k].re, r.c[k].im);
    }
};

struct KS32 {
    using R = float;
    static constexpr bool kScaled = false;
    __device__ __forceinline__ static Colour<R> load(const SpinorView &v, int i, R &w)
    {
        Colour<R> r;
        const float2 *p = static_cast<const float2 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float2 d = __ldg(p + (size_t)k * v.stride);
            r.c[k] = mk(d.x, d.y);
        }
        w = 1.0f;
        return r;
    }
    __device__ __forceinline__ static void store(const SpinorView &v, int i, const Colour<R> &r)
    {
        float2 *p = static_cast<float2 *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) p[(size_t)k * v.stride] = make_float2(r.c[k].re, r.c[k].im);
    }
};

// 16-bit: three 4-byte planes (one complex each); FP16 carries a per-site
// FP32 scale (largest |real component|), returned as the weight w.
template <typename H, bool kNorm>
struct KS16 {
    using R = float;
    static constexpr bool kScaled = kNorm;
    __device__ __forceinline__ static Colour<R> load(const SpinorView &v, int i, R &w)
    {
        Colour<R> r;
        const uint32_t *p = static_cast<const uint32_t *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float2 f = Half16<H>::to2(__ldg(p + (size_t)k * v.stride));
            r.c[k] = mk(f.x, f.y);
        }
        w = kNorm ? __ldg(v.norm + i) : 1.0f;
        return r;
    }
    __device__ __forceinline__ static void store(const SpinorView &v, int i, const Colour<R> &r)
    {
        float inv = 1.0f;
        if (kNorm) {
            float m = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) m = fmaxf(m, fmaxf(fabsf(r.c[k].re), fabsf(r.c[k].im)));
            v.norm[i] = m;
            inv = m > 0.0f ? 1.0f / m : 0.0f;
        }
        uint32_t *p = static_cast<uint32_t *>(v.data) + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) p[(size_t)k * v.stride] = Half16<H>::from2(inv * r.c[k].re, inv * r.c[k].im);
    }
};

template <typename KF, typename GF>
__global__ void __launch_bounds__(128) dslash_ks_kernel(const KsLaunch a)
{
    using R = typename KF::R;
    const int nbp = (a.g.h + 127) / 128;
    const int p = a.both ? (int)(blockIdx.x >= (unsigned)nbp) : a.out_parity;
    const int i = (blockIdx.x - (a.both ? p * nbp : 0)) * blockDim.x + threadIdx.x;
    if (i >= a.g.h) return;
    const Geom &g = a.g;
    const SpinorView &in = a.in[p];
    const SiteCoords c = site_coords(g, i, p);
    const int base = i - c.xh;
    const int fwd = p * 4, bwd = (1 - p) * 4;
    int nb[8];
    const int xf = c.x + 1 == g.L[0] ? 0 : c.x + 1, xb = c.x == 0 ? g.L[0] - 1 : c.x - 1;
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
    // staggered phases of the output site
    const int eta[4] = {1, (c.x & 1) ? -1 : 1, ((c.x + c.y) & 1) ? -1 : 1, ((c.x + c.y + c.z) & 1) ? -1 : 1};
    Colour<R> acc;
#pragma unroll
    for (int a2 = 0; a2 < 3; ++a2) acc.c[a2] = mk((R)0, (R)0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int mu = k >> 1;
        const bool forward = !(k & 1);
        R w;
        const Colour<R> v = KF::load(in, nb[k], w);
        const Link<R> u = GF::load(a.U, (forward ? fwd : bwd) + mu, forward ? i : nb[k]);
        int sgn = eta[mu] * (forward ? 1 : -1);
        if (mu == 3 && anti && (forward ? wf : wb)) sgn = -sgn;
        const R ws = sgn > 0 ? w : -w;
#pragma unroll
        for (int a2 = 0; a2 < 3; ++a2) {
            cx<R> s;
            if (forward) {
                s = cmul(u.m[a2][0], v.c[0]);
                s = cmac(s, u.m[a2][1], v.c[1]);
                s = cmac(s, u.m[a2][2], v.c[2]);
            } else {
                s = cjmul(u.m[0][a2], v.c[0]);
                s = cjmac(s, u.m[1][a2], v.c[1]);
                s = cjmac(s, u.m[2][a2], v.c[2]);
            }
            if (KF::kScaled) {
                acc.c[a2].re = fma(ws, s.re, acc.c[a2].re);
                acc.c[a2].im = fma(ws, s.im, acc.c[a2].im);
            } else {
                acc.c[a2] = sgn > 0 ? acc.c[a2] + s : acc.c[a2] - s;
            }
        }
    }
    KF::store(a.out[p], i, acc);
}

// host [site][3] complex (FP64) <-> device staggered field
template <typename KF>
__global__ void ks_pack_kernel(const FieldView dst, const int parity, const double2 *aos, const Geom g, const int unpack,
                               double2 *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = parity == 2 ? 2 * g.h : g.h;
    if (k >= n) return;
    int half = 0, i = k;
    if (parity == 2) {
        int r = k;
        const int x = r % g.L[0];
        r /= g.L[0];
        const int y = r % g.L[1];
        r /= g.L[1];
        const int z = r % g.L[2];
        const int t = r / g.L[2];
        half = (x + y + z + t) & 1;
        i = k >> 1;
    }
    using R = typename KF::R;
    if (!unpack) {
        Colour<R> v;
#pragma unroll
        for (int a = 0; a < 3; ++a) v.c[a] = mk((R)aos[(size_t)k * 3 + a].x, (R)aos[(size_t)k * 3 + a].y);
        KF::store(dst.hv[half], i, v);
    } else {
        R w;
        const Colour<R> v = KF::load(dst.hv[half], i, w);
#pragma unroll
        for (int a = 0; a < 3; ++a) out[(size_t)k * 3 + a] = make_double2((double)(w * v.c[a].re), (double)(w * v.c[a].im));
    }
}

using GH18 = G16<__half, 18>;
using GH12 = G16<__half, 12>;
using GB18 = G16<__nv_bfloat16, 18>;
using GB12 = G16<__nv_bfloat16, 12>;
using GH8 = G16<__half, 8>;
using GB8 = G16<__nv_bfloat16, 8>;

}  // namespace

#define QCD_KS_CASES(prec, KF, ...)                        \
    switch (prec) {                                        \
    case QCD_PREC_F64: {                                   \
        using KF = KS64;                                   \
        __VA_ARGS__;                                       \
    } break;                                               \
    case QCD_PREC_F32: {                                   \
        using KF = KS32;                                   \
        __VA_ARGS__;                                       \
    } break;                                               \
    case QCD_PREC_F16: {                                   \
        using KF = KS16<__half, true>;                     \
        __VA_ARGS__;                                       \
    } break;                                               \
    case QCD_PREC_BF16: {                                  \
        using KF = KS16<__nv_bfloat16, false>;             \
        __VA_ARGS__;                                       \
    } break;                                               \
    default:                                               \
        return cudaErrorInvalidValue;                      \
    }

cudaError_t launch_dslash_ks(int prec, int recon, const KsLaunch &a, cudaStream_t s)
{
    const dim3 grid((a.g.h + 127) / 128 * (a.both ? 2 : 1)), block(128);
    if (recon != 18 && recon != 12 && recon != 8) return cudaErrorInvalidValue;
    const int r = recon;
    switch (prec) {
    case QCD_PREC_F64:
        if (r == 18) dslash_ks_kernel<KS64, GF64<18>><<<grid, block, 0, s>>>(a);
        else if (r == 12) dslash_ks_kernel<KS64, GF64<12>><<<grid, block, 0, s>>>(a);
        else dslash_ks_kernel<KS64, GF64<8>><<<grid, block, 0, s>>>(a);
        break;
    case QCD_PREC_F32:
        if (r == 18) dslash_ks_kernel<KS32, GF32<18>><<<grid, block, 0, s>>>(a);
        else if (r == 12) dslash_ks_kernel<KS32, GF32<12>><<<grid, block, 0, s>>>(a);
        else dslash_ks_kernel<KS32, GF32<8>><<<grid, block, 0, s>>>(a);
        break;
    case QCD_PREC_F16:
        if (r == 18) dslash_ks_kernel<KS16<__half, true>, GH18><<<grid, block, 0, s>>>(a);
        else if (r == 12) dslash_ks_kernel<KS16<__half, true>, GH12><<<grid, block, 0, s>>>(a);
        else dslash_ks_kernel<KS16<__half, true>, GH8><<<grid, block, 0, s>>>(a);
        break;
    case QCD_PREC_BF16:
        if (r == 18) dslash_ks_kernel<KS16<__nv_bfloat16, false>, GB18><<<grid, block, 0, s>>>(a);
        else if (r == 12) dslash_ks_kernel<KS16<__nv_bfloat16, false>, GB12><<<grid, block, 0, s>>>(a);
        else dslash_ks_kernel<KS16<__nv_bfloat16, false>, GB8><<<grid, block, 0, s>>>(a);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_ks_pack(const FieldView &f, int parity, const double2 *aos, const Geom &g, cudaStream_t s)
{
    const int n = parity == 2 ? 2 * g.h : g.h;
    QCD_KS_CASES(f.prec, KF, ks_pack_kernel<KF><<<(n + 127) / 128, 128, 0, s>>>(f, parity, aos, g, 0, nullptr));
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_ks_unpack(double2 *aos, const FieldView &f, int parity, const Geom &g, cudaStream_t s)
{
    const int n = parity == 2 ? 2 * g.h : g.h;
    QCD_KS_CASES(f.prec, KF, ks_pack_kernel<KF><<<(n + 127) / 128, 128, 0, s>>>(f, parity, nullptr, g, 1, aos));
    note_launches();
    return cudaGetLastError();
}

}  // namespace qcd
