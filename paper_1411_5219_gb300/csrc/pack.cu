// Layout conversion between the host form (FP64, array of structures,
// lexicographic sites) and the device form (structure of arrays per parity,
// in the storage precision; CL2QCD arXiv:1411.5219 Sec. 4 keeps device
// buffers in SoA form because GPUs need it for coalesced access), plus the
// conversion of a gauge field between device formats.
#include <cstring>

#include "qcd_ops.h"

namespace qcd {

namespace {

template <typename R2, typename R1>
__device__ __forceinline__ Link<R2> cvt_link(const Link<R1> &a)
{
    Link<R2> b;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) b.m[i][j] = mk((R2)a.m[i][j].re, (R2)a.m[i][j].im);
    return b;
}

struct LexCoords {
    int parity;
    int half;  // lex / 2
};
__device__ __forceinline__ LexCoords lex_coords(const Geom &g, int lex)
{
    int r = lex;
    const int x = r % g.L[0];
    r /= g.L[0];
    const int y = r % g.L[1];
    r /= g.L[1];
    const int z = r % g.L[2];
    const int t = r / g.L[2];
    return LexCoords{(x + y + z + t) & 1, lex >> 1};
}

template <typename GF>
__global__ void gauge_pack_kernel(const GaugeView dst, const double2 *aos, const Geom g)
{
    const int lex = blockIdx.x * blockDim.x + threadIdx.x;
    if (lex >= 2 * g.h) return;
    const LexCoords c = lex_coords(g, lex);
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
        Link<double> u;
        const double2 *src = aos + ((size_t)lex * 4 + mu) * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) u.m[k / 3][k % 3] = mk(src[k].x, src[k].y);
        GF::store64(dst, c.parity * 4 + mu, c.half, u);
    }
}

template <typename GO, typename GI>
__global__ void gauge_convert_kernel(const GaugeView dst, const GaugeView src, const int h)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= h) return;
    GO::store64(dst, b, i, cvt_link<double>(GI::load(src, b, i)));
}

// Largest |entry error| of the links stored in format GF against the FP64
// reference, over the grid (atomicMax on the bit pattern, which orders
// non-negative doubles; a non-finite error counts as 1e300).
template <typename R>
__device__ __forceinline__ double link_max_err(const Link<R> &v, const Link<double> &u)
{
    double m = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            double e = fmax(fabs((double)v.m[a][b].re - u.m[a][b].re), fabs((double)v.m[a][b].im - u.m[a][b].im));
            if (!(e < 1e300)) e = 1e300;
            m = fmax(m, e);
        }
    return m;
}
__device__ __forceinline__ void max_into(unsigned long long *out, double e)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e = fmax(e, __shfl_xor_sync(0xffffffffu, e, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(e));
}

template <typename GF>
__global__ void gauge_check_aos_kernel(const GaugeView dst, const double2 *aos, const Geom g, unsigned long long *out)
{
    const int lex = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (lex < 2 * g.h) {
        const LexCoords c = lex_coords(g, lex);
        for (int mu = 0; mu < 4; ++mu) {
            Link<double> u;
            const double2 *src = aos + ((size_t)lex * 4 + mu) * 9;
#pragma unroll
            for (int k = 0; k < 9; ++k) u.m[k / 3][k % 3] = mk(src[k].x, src[k].y);
            e = fmax(e, link_max_err(GF::load(dst, c.parity * 4 + mu, c.half), u));
        }
    }
    max_into(out, e);
}

template <typename GO, typename GI>
__global__ void gauge_check_kernel(const GaugeView dst, const GaugeView src, const int h, unsigned long long *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    double e = 0.0;
    if (i < h) e = link_max_err(GO::load(dst, b, i), cvt_link<double>(GI::load(src, b, i)));
    max_into(out, e);
}

template <typename SF>
__device__ __forceinline__ void store_site(const FieldView &f, int half, int i, const Spinor<double> &v)
{
    Spinor<typename SF::R> w;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) w.c[s][c] = mk((typename SF::R)v.c[s][c].re, (typename SF::R)v.c[s][c].im);
    SF::store(f.hv[half], i, w);
}

template <typename SF>
__global__ void spinor_pack_kernel(const FieldView dst, const int parity, const double2 *aos, const Geom g)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = parity == 2 ? 2 * g.h : g.h;
    if (k >= n) return;
    Spinor<double> v;
    const double2 *src = aos + (size_t)k * 12;
#pragma unroll
    for (int j = 0; j < 12; ++j) v.c[j / 3][j % 3] = mk(src[j].x, src[j].y);
    if (parity == 2) {
        const LexCoords c = lex_coords(g, k);
        store_site<SF>(dst, c.parity, c.half, v);
    } else {
        store_site<SF>(dst, 0, k, v);
    }
}

template <typename SF>
__global__ void spinor_unpack_kernel(double2 *aos, const FieldView src, const int parity, const Geom g)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = parity == 2 ? 2 * g.h : g.h;
    if (k >= n) return;
    int half = 0, i = k;
    if (parity == 2) {
        const LexCoords c = lex_coords(g, k);
        half = c.parity;
        i = c.half;
    }
    const Spinor<typename SF::R> w = SF::load(src.hv[half], i);
    double2 *d = aos + (size_t)k * 12;
#pragma unroll
    for (int j = 0; j < 12; ++j) d[j] = make_double2((double)w.c[j / 3][j % 3].re, (double)w.c[j / 3][j % 3].im);
}

}  // namespace

#define QCD_G_CASES(prec, recon, GF, ...)                                     \
    if (prec == QCD_PREC_F64 && recon == 18) {                                \
        using GF = GF64<18>;                                                  \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_F64 && recon == 12) {                         \
        using GF = GF64<12>;                                                  \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_F32 && recon == 18) {                         \
        using GF = GF32<18>;                                                  \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_F32 && recon == 12) {                         \
        using GF = GF32<12>;                                                  \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_F16 && recon == 18) {                         \
        using GF = G16<__half, 18>;                                           \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_F16 && recon == 12) {                         \
        using GF = G16<__half, 12>;                                           \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_BF16 && recon == 18) {                        \
        using GF = G16<__nv_bfloat16, 18>;                                    \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_BF16 && recon == 12) {                        \
        using GF = G16<__nv_bfloat16, 12>;                                    \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_F64 && recon == 8) {                          \
        using GF = GF64<8>;                                                   \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_F32 && recon == 8) {                          \
        using GF = GF32<8>;                                                   \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_F16 && recon == 8) {                          \
        using GF = G16<__half, 8>;                                            \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_BF16 && recon == 8) {                         \
        using GF = G16<__nv_bfloat16, 8>;                                     \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_DF64 && recon == 18) {                        \
        using GF = GDF64<18>;                                                 \
        __VA_ARGS__;                                                          \
    } else if (prec == QCD_PREC_DF64 && recon == 12) {                        \
        using GF = GDF64<12>;                                                 \
        __VA_ARGS__;                                                          \
    } else {                                                                  \
        return cudaErrorInvalidValue;                                         \
    }

#define QCD_SP_CASES2(prec, SF, ...)      \
    switch (prec) {                       \
    case QCD_PREC_F64: {                  \
        using SF = SpF64;                 \
        __VA_ARGS__;                      \
    } break;                              \
    case QCD_PREC_F32: {                  \
        using SF = SpF32;                 \
        __VA_ARGS__;                      \
    } break;                              \
    case QCD_PREC_F16: {                  \
        using SF = SpF16;                 \
        __VA_ARGS__;                      \
    } break;                              \
    case QCD_PREC_BF16: {                 \
        using SF = SpBF16;                \
        __VA_ARGS__;                      \
    } break;                              \
    case QCD_PREC_DF64: {                 \
        using SF = SpDF64;                \
        __VA_ARGS__;                      \
    } break;                              \
    default:                              \
        return cudaErrorInvalidValue;     \
    }

cudaError_t launch_gauge_pack(const GaugeView &dst, int prec, int recon, const double2 *aos, const Geom &g,
                              cudaStream_t s)
{
    const int n = 2 * g.h;
    QCD_G_CASES(prec, recon, GF, gauge_pack_kernel<GF><<<(n + 127) / 128, 128, 0, s>>>(dst, aos, g));
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_gauge_convert(const GaugeView &dst, int dprec, int drecon, const GaugeView &src, int sprec,
                                 int srecon, const Geom &g, cudaStream_t s)
{
    const dim3 grid((g.h + 127) / 128, 8);
    QCD_G_CASES(dprec, drecon, GO,
                QCD_G_CASES(sprec, srecon, GI, gauge_convert_kernel<GO, GI><<<grid, 128, 0, s>>>(dst, src, g.h)));
    note_launches();
    return cudaGetLastError();
}

// Largest entry error of a reconstruct-8 field `dst` against its FP64
// source: the host array staged at `aos` (when not null) or the device
// field `src` in format (sprec, srecon).  Synchronises the stream.
cudaError_t gauge_recon8_error(const GaugeView &dst, int prec, const double2 *aos, const GaugeView &src, int sprec,
                               int srecon, const Geom &g, cudaStream_t s, double *max_err)
{
    unsigned long long *d = nullptr, hbits = 0;
    cudaError_t e = cudaMallocAsync(&d, sizeof(*d), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(d, 0, sizeof(*d), s);
    if (e == cudaSuccess) {
        e = [&]() -> cudaError_t {
            if (aos) {
                QCD_G_CASES(prec, 8, GF, gauge_check_aos_kernel<GF><<<(2 * g.h + 127) / 128, 128, 0, s>>>(dst, aos, g, d));
            } else {
                const dim3 grid((g.h + 127) / 128, 8);
                QCD_G_CASES(prec, 8, GO,
                            QCD_G_CASES(sprec, srecon, GI, gauge_check_kernel<GO, GI><<<grid, 128, 0, s>>>(dst, src, g.h, d)));
            }
            return cudaSuccess;
        }();
        note_launches();
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbits, d, sizeof(hbits), cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    double v;
    memcpy(&v, &hbits, sizeof(v));
    *max_err = v;
    return e;
}

cudaError_t launch_spinor_pack(const FieldView &dst, int parity, const double2 *aos, const Geom &g, cudaStream_t s)
{
    const int n = parity == 2 ? 2 * g.h : g.h;
    QCD_SP_CASES2(dst.prec, SF, spinor_pack_kernel<SF><<<(n + 127) / 128, 128, 0, s>>>(dst, parity, aos, g));
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_spinor_unpack(double2 *aos, const FieldView &src, int parity, const Geom &g, cudaStream_t s)
{
    const int n = parity == 2 ? 2 * g.h : g.h;
    QCD_SP_CASES2(src.prec, SF, spinor_unpack_kernel<SF><<<(n + 127) / 128, 128, 0, s>>>(aos, src, parity, g));
    note_launches();
    return cudaGetLastError();
}

}  // namespace qcd
