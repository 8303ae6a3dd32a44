// Time-slab domain decomposition: the face pack and unpack kernels.
//
// The paper splits the lattice in the time direction when one device is
// not enough (Sec. 7).  A rank holds Lt_loc consecutive time slices of the
// global lattice on an extended local lattice of Lt_loc + 2 slices (created
// with t_bc = +1): slices 1 .. Lt_loc are its own, slice 0 and slice
// Lt_loc + 1 are halos filled from the neighbouring ranks.  Only the t hops
// of the first and last own slice reach a halo, and they need half as many
// numbers as a full spinor:
//
//   to the previous rank (its forward t hops): h = psi_up - S psi_dn, the
//     projected half spinor of this rank's first slice (gamma_t = [[0,1],
//     [1,0]] in the chiral basis, S = +1 for D, -1 for D^dagger);
//   to the next rank (its backward t hops): u = U_t(x)^dagger (psi_up +
//     S psi_dn), projected and multiplied by this rank's last t links.
//
// Six complex numbers per face site (96 bytes in FP64).  The receiver writes
// a face into its halo slice as a spinor with upper spins = face and lower
// spins = 0 (the t links of the backward halo slice are the identity), so
// the unchanged hopping kernel projects, multiplies and rebuilds exactly
// what the unsplit kernel would (the projection of (h, 0) is h; 1 times u is
// u).  The factor of the global antiperiodic boundary is applied by the
// sender whose face crosses it.  Exchange of the faces between ranks (NCCL,
// peer copies or host transfers into the receiver's own buffer) is the
// caller's; the library only packs and unpacks device buffers.
#include "qcd_handles.h"

namespace qcd {
namespace {

// face[k * n + j], k = 3 s + c (spin s = 0, 1 of the half spinor, colour c)
__global__ void __launch_bounds__(kThreads) face_pack_kernel(const SpinorView in, const GaugeView U, int parity,
                                                             int slice, int st, int to_next, double s_proj,
                                                             double sign, double2 *face)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= st) return;
    const int i = slice * st + j;
    const Spinor<double> psi = SpF64::load(in, i);
    HalfSpinor<double> h;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cx<double> a = psi.c[s][c], b = psi.c[2 + s][c];
            h.c[s][c] = mk(fma(-s_proj, b.re, a.re), fma(-s_proj, b.im, a.im));
        }
    if (to_next) {
        // u = U_t(x)^dagger h, x this site (block (parity, t))
        const Link<double> u = GF64<18>::load(U, parity * 4 + 3, i);
        HalfSpinor<double> v;
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                cx<double> w = cjmul(u.m[0][a], h.c[s][0]);
                w = cjmac(w, u.m[1][a], h.c[s][1]);
                w = cjmac(w, u.m[2][a], h.c[s][2]);
                v.c[s][a] = w;
            }
        h = v;
    }
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) face[(size_t)(3 * s + c) * st + j] = make_double2(sign * h.c[s][c].re, sign * h.c[s][c].im);
}

__global__ void __launch_bounds__(kThreads) face_unpack_kernel(const SpinorView out, int slice, int st,
                                                               const double2 *face)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= st) return;
    Spinor<double> v;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 f = face[(size_t)(3 * s + c) * st + j];
            v.c[s][c] = mk(f.x, f.y);
            v.c[2 + s][c] = mk(0.0, 0.0);
        }
    SpF64::store(out, slice * st + j, v);
}

}  // namespace
}  // namespace qcd

using namespace qcd;

extern "C" qcd_status qcd_face_pack(const qcd_gauge *g, const qcd_spinor *in, int face, int dagger, double sign,
                                    double *face_dev, void *stream)
{
    if (!g || !in || !face_dev) return fail(QCD_ERR_INVALID_ARG, "face_pack: NULL argument");
    if (face != QCD_FACE_TO_PREV && face != QCD_FACE_TO_NEXT) return fail(QCD_ERR_INVALID_ARG, "face_pack: bad face");
    if (in->lat != g->lat || in->parity == QCD_PARITY_FULL || in->prec != QCD_PREC_F64 || in->ks)
        return fail(QCD_ERR_INVALID_ARG, "face_pack: in must be an EVEN or ODD F64 Wilson field on the gauge's lattice");
    if (g->prec != QCD_PREC_F64) return fail(QCD_ERR_INVALID_ARG, "face_pack: the gauge field must be F64");
    const qcd_lattice *lat = g->lat;
    const int T = lat->dims[3];
    if (T < 4 || lat->t_bc != 1)
        return fail(QCD_ERR_INVALID_ARG, "face_pack: an extended slab lattice has t_bc = +1 and >= 4 time slices");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    qcd_status st = QCD_OK;
    const GaugeView U = gauge_view(g, QCD_PREC_F64, 18, s, &st);
    if (st != QCD_OK) return st;
    const int n = lat->geom.st;  // sites of one parity in one time slice
    const double s_proj = face == QCD_FACE_TO_PREV ? (dagger ? -1.0 : 1.0) : (dagger ? 1.0 : -1.0);
    const int slice = face == QCD_FACE_TO_PREV ? 1 : T - 2;
    const FieldView v = view_of(in);
    face_pack_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(v.hv[0], U, in->parity, slice, n,
                                                                       face == QCD_FACE_TO_NEXT, s_proj, sign,
                                                                       reinterpret_cast<double2 *>(face_dev));
    note_launches();
    return check_cuda(cudaGetLastError(), "face_pack");
}

extern "C" qcd_status qcd_face_unpack(qcd_spinor *out, int face, const double *face_dev, void *stream)
{
    if (!out || !face_dev) return fail(QCD_ERR_INVALID_ARG, "face_unpack: NULL argument");
    if (face != QCD_FACE_FROM_PREV && face != QCD_FACE_FROM_NEXT) return fail(QCD_ERR_INVALID_ARG, "face_unpack: bad face");
    if (out->parity == QCD_PARITY_FULL || out->prec != QCD_PREC_F64 || out->ks)
        return fail(QCD_ERR_INVALID_ARG, "face_unpack: out must be an EVEN or ODD F64 Wilson field");
    const qcd_lattice *lat = out->lat;
    const int T = lat->dims[3];
    if (T < 4 || lat->t_bc != 1)
        return fail(QCD_ERR_INVALID_ARG, "face_unpack: an extended slab lattice has t_bc = +1 and >= 4 time slices");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = lat->geom.st;
    const int slice = face == QCD_FACE_FROM_PREV ? 0 : T - 1;
    const FieldView v = view_of(out);
    face_unpack_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(v.hv[0], slice, n,
                                                                         reinterpret_cast<const double2 *>(face_dev));
    note_launches();
    return check_cuda(cudaGetLastError(), "face_unpack");
}
