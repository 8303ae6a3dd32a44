/*
 * libqcd: GB300 (sm_103a) even-odd Wilson / twisted-mass Wilson operator and
 * CG solver, C ABI.
 *
 * The paper (CL2QCD, arXiv:1411.5219) names the most expensive part of a
 * lattice QCD simulation as the inversion of the fermion matrix, D phi = psi,
 * by a Krylov method such as CG, in which the product D phi -- dominated by
 * its hopping part, the "Dslash" -- is applied many times and is limited by
 * memory bandwidth (Sec. 1).  It implements Wilson and twisted-mass Wilson
 * fermions (Sec. 3), on structure-of-arrays device buffers (Sec. 4), in
 * double precision (Sec. 4).  This library provides that hot path:
 *
 *   D_hop psi(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                         + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu) ]
 *   M = A - kappa D_hop,   A = 1 + i a gamma_5,   a = 2 kappa mu
 *
 * with gamma matrices in the chiral basis (gamma_k = [[0, -i sigma_k],
 * [i sigma_k, 0]], gamma_4 = [[0, 1], [1, 0]], gamma_5 = diag(1,1,-1,-1)),
 * periodic boundaries in space and the factor t_bc on hops that wrap in
 * time.  The paper gives no formulas; these conventions are the standard
 * ones.  Even-odd preconditioning and mixed precision are not in the paper;
 * they are the usual way to run this inversion fast:
 *
 *   Mhat = A - kappa^2 D_eo A^-1 D_oe   on even sites (Schur complement),
 *   A^-1 = (1 - i a gamma_5) / (1 + a^2).
 *
 * Sites: lex = x + Lx*(y + Ly*(z + Lz*t)); parity p = (x+y+z+t) mod 2.  A
 * half field holds the sites of one parity; its host form is
 * parity-compacted, site lex at index lex/2.
 *
 * Host layouts (interleaved re/im doubles, C order):
 *   gauge   [t][z][y][x][mu][a][b]   (mu = 0..3 for x, y, z, t; U_mu(x)[a][b])
 *   spinor  [t][z][y][x][spin][colour]        full field, 24 doubles per site
 *   half    [lex/2][spin][colour]             one parity, 24 doubles per site
 *
 * Conventions of every call:
 *   - Returns a qcd_status; no C++ exception crosses the ABI.
 *     qcd_last_error() gives a message for the last failure on this thread.
 *   - `stream` is a cudaStream_t (NULL: the legacy default stream).  Calls
 *     are asynchronous on it unless stated otherwise; host buffers passed to
 *     upload/download must stay valid until the stream reaches the copy
 *     (the call returns only after the copy when the buffer is pageable).
 *   - The library owns every handle and the device memory it allocates;
 *     destroy each handle once; destroying NULL is a no-op.  A handle must
 *     outlive the work queued on it.
 *   - Work on handles of the same lattice must be ordered on one stream:
 *     a lattice handle owns the scratch (reductions, staging, solver
 *     fields) that these calls share.
 */
#ifndef QCD_H
#define QCD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int qcd_status;
#define QCD_OK 0
#define QCD_ERR_INVALID_ARG 1   /* bad handle, size, layout or parameter */
#define QCD_ERR_OOM 2           /* device allocation failed */
#define QCD_ERR_CUDA 3          /* a CUDA call failed */
#define QCD_ERR_NOT_CONVERGED 4 /* maxiter reached; x and stats still written */
#define QCD_ERR_BREAKDOWN 5     /* CG breakdown: <p,Ap> <= 0 or non-finite values */
#define QCD_ERR_TIMEOUT 6       /* reserved for bounded device waits */
#define QCD_ERR_CANCELLED 7     /* a queued server request dropped by qcd_server_destroy */

/* Storage precision of a field.  F64/F32/F16/BF16 are IEEE formats (F16
 * spinors carry an FP32 per-site scale).  DF64 ("double-float") stores each
 * real as the unevaluated sum hi + lo of two FP32 numbers (8 bytes, ~48
 * significant bits) and its kernels compute in pairs of FP32 numbers with
 * error-free transformations: FP64-accurate to ~1e-14 at FP32 instruction
 * rates, since GB300 runs FP32 58x faster than FP64.  The paper computes all
 * in double precision (Sec. 4); DF64 is this library's way to do so on
 * GB300 and is always labelled as such. */
typedef enum { QCD_PREC_F64 = 0, QCD_PREC_F32 = 1, QCD_PREC_F16 = 2, QCD_PREC_BF16 = 3, QCD_PREC_DF64 = 4 } qcd_prec;
/* Link storage: 18 reals (full matrix), 12 (rows 0 and 1; row 2 is
 * rebuilt as conj(row0 x row1), exact for SU(3)) or 8.  Reconstruct-8 is
 * pivoted for links near the identity: with W = U with its columns
 * reversed, it stores W_00, W_01, W_10 and tan(arg/2) of W_02 = U_00 and
 * W_20 = U_22; the two magnitudes follow from unit norms, the rest from
 * unitarity and det U = 1, dividing by |W_01|^2 + |W_02|^2 (close to 1 when
 * the diagonal dominates).  Every field written in this form is checked
 * against its FP64 source (which synchronises the stream) and refused with
 * INVALID_ARG when an entry is off by more than 1e-13 (F64), 32 u (F32) or
 * 4 u (F16, BF16), u the unit roundoff; DF64 takes 18 only. */
typedef enum { QCD_RECON_18 = 18, QCD_RECON_12 = 12, QCD_RECON_8 = 8 } qcd_recon;
typedef enum { QCD_PARITY_EVEN = 0, QCD_PARITY_ODD = 1, QCD_PARITY_FULL = 2 } qcd_parity;

typedef struct qcd_lattice qcd_lattice;
typedef struct qcd_gauge qcd_gauge;
typedef struct qcd_spinor qcd_spinor;

/* Name of a status code (static string). */
const char *qcd_status_string(qcd_status s);
/* Message of the last failing call on this thread (static, thread-local). */
const char *qcd_last_error(void);
/* Library version string. */
const char *qcd_version(void);
/* Block the calling thread until all work queued on `stream` is done.
 * Errors: CUDA (a failure of earlier asynchronous work is reported here). */
qcd_status qcd_stream_sync(void *stream);

/* ---------------------------------------------------------------- lattice */

/* A lattice Lx x Ly x Lz x Lt on the current CUDA device.  dims[mu] must
 * be even and >= 2 (even-odd indexing needs even Lx; the boundary factor
 * needs even extents for a consistent parity).  t_bc = +1 (periodic) or -1
 * (antiperiodic) in time (Sec. 1 discretises space-time on an Ns^3 x Nt
 * hypercube).  Its device state (CG state, reduction counters) is zeroed
 * before the call returns, so any stream may use the lattice at once; the
 * call waits for the legacy default stream.  Errors: INVALID_ARG for bad
 * extents or a volume too large for 32-bit site indices; OOM. */
qcd_status qcd_lattice_create(const int dims[4], int t_bc, qcd_lattice **out);
/* Release the lattice.  Gauge fields and spinors created on it keep it
 * alive: its memory is freed when the last of them is destroyed, so fields
 * and their lattice may be destroyed in any order.  NULL is a no-op. */
void qcd_lattice_destroy(qcd_lattice *lat);

/* ------------------------------------------------------------------ gauge */

/* A gauge field U_mu(x) in SU(3) (4 links per site, Sec. 1 and 4), stored
 * on the device per (parity, mu) block, site-fastest (SoA, Sec. 4), in
 * precision `prec` and with `recon` reals per link.  The field also keeps
 * derived copies in other precisions, made on the device from this one on
 * first use by a Dslash of that precision.  The field is zero when the
 * call returns (it waits for the legacy default stream).  Errors:
 * INVALID_ARG; OOM; CUDA. */
qcd_status qcd_gauge_create(const qcd_lattice *lat, qcd_prec prec, qcd_recon recon, qcd_gauge **out);
/* Copy a host gauge field (host layout above, 4*V*9 complex doubles) to
 * the device and convert it; drops derived copies.  Recon-12 and recon-8
 * assume SU(3) links.  Errors: INVALID_ARG (NULL; recon-8 links out of
 * reach, see qcd_recon); CUDA. */
qcd_status qcd_gauge_upload(qcd_gauge *g, const double *host, void *stream);
/* Build (if missing) the derived copy used by kernels of precision
 * `prec` with `recon` reals per link.  Optional: calls build it on first
 * use, outside stream capture (a new copy is complete, its stream
 * synchronised, before any stream may read it; a call on a capturing stream
 * that needs a missing copy fails with INVALID_ARG).  Errors: INVALID_ARG
 * (also recon-8 links out of reach); OOM. */
qcd_status qcd_gauge_prepare(qcd_gauge *g, qcd_prec prec, qcd_recon recon, void *stream);
void qcd_gauge_destroy(qcd_gauge *g);

/* ----------------------------------------------------------------- spinor */

/* A spinor (fermion) field, 4 spins x 3 colours per site (Sec. 4), on one
 * parity (EVEN/ODD, V/2 sites) or on all sites (FULL = even half then odd
 * half).  F16 keeps one FP32 scale per site.  The field is zero when the
 * call returns, so an upload on any stream, blocking or not, is not
 * overwritten later (the call waits for the legacy default stream).
 * Errors: INVALID_ARG; OOM. */
qcd_status qcd_spinor_create(const qcd_lattice *lat, qcd_parity parity, qcd_prec prec, qcd_spinor **out);
/* A staggered field (one colour vector, 3 complex per site), the field of
 * the paper's second Dirac operator D_KS (Sec. 1, Sec. 6), in F64, F32, F16
 * (with FP32 per-site scale) or BF16.  Host layout [t][z][y][x][colour]
 * (FULL) or [lex/2][colour] (EVEN/ODD); qcd_spinor_upload/download and
 * qcd_spinor_destroy accept it, the Wilson operators, norms, conversions
 * and solvers reject it (INVALID_ARG).  Errors: INVALID_ARG; OOM. */
qcd_status qcd_spinor_create_ks(const qcd_lattice *lat, qcd_parity parity, qcd_prec prec, qcd_spinor **out);
/* Device bytes of such a field: *data_bytes for the planes, *norm_bytes
 * for the F16 per-site scales (0 otherwise). */
qcd_status qcd_spinor_bytes(const qcd_lattice *lat, qcd_parity parity, qcd_prec prec, size_t *data_bytes,
                            size_t *norm_bytes);
/* A spinor handle over caller-owned device memory of at least the sizes
 * qcd_spinor_bytes reports (256-byte aligned); the library never frees
 * it.  `norm` is required for F16 only. */
qcd_status qcd_spinor_wrap_device(const qcd_lattice *lat, qcd_parity parity, qcd_prec prec, void *data, void *norm,
                                  qcd_spinor **out);
/* Host (FP64, host layout above; FULL: V*12 complex, EVEN/ODD: V/2*12
 * complex) to device, converting to the field's precision. */
qcd_status qcd_spinor_upload(qcd_spinor *s, const double *host, void *stream);
/* Device to host (FP64, same layouts).  Asynchronous: synchronise the
 * stream before reading `host`. */
qcd_status qcd_spinor_download(const qcd_spinor *s, double *host, void *stream);
/* Set to zero. */
qcd_status qcd_spinor_zero(qcd_spinor *s, void *stream);
/* Copy with precision conversion between fields of the same lattice and
 * parity. */
qcd_status qcd_spinor_convert(qcd_spinor *dst, const qcd_spinor *src, void *stream);
/* result[0] = sum |s|^2 over the field's sites, FP64 accumulation, fixed
 * summation order.  `result` is a device pointer to 1 double; the value is
 * ready when the stream reaches it.  Uses the lattice's reduction scratch. */
qcd_status qcd_spinor_norm2(const qcd_spinor *s, double *result_device, void *stream);
void qcd_spinor_destroy(qcd_spinor *s);

/* out[k] = D_hop in[k] (dagger: D_hop^dagger in[k]) for k < nrhs (1..32): the
 * same parity rules as qcd_apply_dslash, all fields of one precision.  The
 * right-hand sides are gathered into one batched field (the rhs index
 * fastest inside each plane) so that a single launch reads each link once
 * for all of them; the results are scattered back.  Errors: INVALID_ARG;
 * OOM; CUDA. */
qcd_status qcd_apply_dslash_multi(const qcd_gauge *g, qcd_spinor *const *out, const qcd_spinor *const *in, int nrhs,
                                  int dagger, void *stream);

/* |x|^2 = sum_i x[i]^2 of n doubles at x_device (e.g. the planes of an F64
 * spinor field), written to result_device (1 double), in FP64 with a fixed
 * summation order -- the reduction of qcd_spinor_norm2 without any
 * allocation.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory (a host framework that has
 * reserved all device memory for its own allocator, or a latency-critical
 * path that cannot accept cudaMalloc's implicit device synchronisation).
 * It needs no lattice or spinor handle and calls no cudaMalloc or cudaFree:
 * its scratch (8192 partial sums and a ticket counter, 64 KiB) is a static
 * device array that every GPU loading the library holds until exit, which
 * limits n to 16,777,216 doubles; larger n returns INVALID_ARG.  The first
 * call on a device looks up that array's device address (make it before
 * any stream capture).  All calls on a device share the array: calls that
 * overlap on the GPU (different streams, no ordering) race; each call
 * clears the counter before it launches.  n = 0 writes 0.  Errors:
 * INVALID_ARG (NULL pointers, n too large); CUDA. */
qcd_status qcd_norm2_noalloc(const double *x_device, size_t n, double *result_device, void *stream);

/* -------------------------------------------------------------- operators */

/* out = D_hop in (dagger = 0) or D_hop^dagger in (dagger = 1): the Dslash
 * (Sec. 1 and 6).  With out of parity p (EVEN or ODD) and in of parity 1-p
 * this is the block D_eo (p = EVEN) or D_oe (p = ODD); with both FULL it is
 * the hopping term on the whole lattice.  out and in share the precision
 * (F64: FP64 arithmetic; F32/F16/BF16: FP32 arithmetic); the gauge field's
 * copy in that precision and with the gauge field's recon is used.
 * Errors: INVALID_ARG (parities, lattices, precisions); CUDA. */
qcd_status qcd_apply_dslash(const qcd_gauge *g, qcd_spinor *out, const qcd_spinor *in, int dagger, void *stream);

/* out = D_KS in, the staggered derivative (Sec. 1, Sec. 6):
 *   (D_KS chi)(x) = sum_mu eta_mu(x) [U_mu(x) chi(x+mu) - U_mu(x-mu)^dagger chi(x-mu)],
 *   eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z),
 * with t_bc on hops that wrap in time; 570 flop per site, as the paper
 * counts (no factor 1/2).  Staggered fields of one precision; parities as
 * for qcd_apply_dslash (D_KS connects even and odd sites only).  The gauge
 * field's copy in that precision and recon is used.  D_KS^dagger = -D_KS.
 * Errors: INVALID_ARG; CUDA. */
qcd_status qcd_apply_dslash_ks(const qcd_gauge *g, qcd_spinor *out, const qcd_spinor *in, void *stream);

/* eo = 0: out = M in on FULL fields, M = A - kappa D_hop (Wilson, Sec. 3;
 *         twisted mass for mu != 0, Sec. 3).
 * eo = 1: out = Mhat in on EVEN fields (Schur complement above).
 * dagger = 1 applies the adjoint (M^dagger = A^dagger - kappa D_hop^dagger).
 * F64 fields only.  Errors: INVALID_ARG; CUDA. */
qcd_status qcd_apply_M(const qcd_gauge *g, qcd_spinor *out, const qcd_spinor *in, double kappa, double mu, int eo,
                       int dagger, void *stream);

/* ----------------------------------------------------------------- solver */

typedef struct {
    double kappa;          /* hopping parameter */
    double mu;             /* twisted mass (0: Wilson) */
    double tol;            /* target relative residual (e.g. 1e-10) */
    int maxiter;           /* CG iteration cap, 1 .. 2^30 */
    int eo;                /* 1: even-odd Schur complement (solves M x = b) */
    int normal;            /* eo = 0 only: 1 solves M^dagger M x = b, 0 solves M x = b (CGNR) */
    qcd_prec inner_prec;   /* F64: plain FP64 CG; F32/F16/BF16/DF64: inner iterations in that precision with FP64
                              reliable updates (DF64 accumulates its correction in DF64, the others in FP32) */
    qcd_recon inner_recon; /* link storage of the inner (sloppy) operator (DF64 always uses 18) */
    double reliable_delta; /* mixed: reliable update when |r| < delta * max|r| since the last one, in (0, 1);
                              0 chooses by inner precision: F32 1e-3, F16 1e-2, BF16 0.1, DF64 1e-4 */
} qcd_solver_params;

typedef struct {
    int iterations;            /* CG iterations */
    int reliable_updates;      /* FP64 true-residual recomputations */
    double true_rel_residual;  /* |rhs - A x| / |rhs| of the CG system, FP64 */
    double full_rel_residual;  /* |b - M x| / |b| (normal: |b - M^dag M x| / |b|), FP64 */
    double seconds;            /* wall time of the call */
} qcd_solver_stats;

/* Solve for x (FULL, F64) given b (FULL, F64) by conjugate gradient (Sec. 1):
 *   eo = 1:  b'_e = b_e + kappa D_eo A^-1 b_o;  CG on Mhat^dag Mhat x_e =
 *            Mhat^dag b'_e;  x_o = A^-1 (b_o + kappa D_oe x_e).
 *   eo = 0:  CG on M^dag M x = b (normal = 1) or = M^dag b (normal = 0).
 * Stops when the iterated residual reaches tol relative to the CG right-hand
 * side and the FP64 true residual confirms it (otherwise it restarts the
 * residual and continues).  Mixed precision runs the inner iterations on
 * fields and links of `inner_prec` (FP32 arithmetic), accumulates x in FP64
 * and replaces the residual by the FP64 true residual at each reliable
 * update.  Blocks until the solve is done.  Returns OK, NOT_CONVERGED
 * (maxiter; x and stats written), BREAKDOWN, INVALID_ARG, OOM or CUDA. */
qcd_status qcd_solve_cg(const qcd_gauge *g, qcd_spinor *x, const qcd_spinor *b, const qcd_solver_params *params,
                        qcd_solver_stats *stats, void *stream);

/* nrhs (1..32) systems with the same gauge field and parameters, solved by
 * one batched CG (the spec batching of many sources): every hopping
 * launch reads each link once for all right-hand sides; each system keeps
 * its own alpha, beta and convergence and stops changing once its FP64 true
 * residual meets tol.  x[k], b[k] as for qcd_solve_cg; stats[k] per system
 * (iterations = the iteration at which system k was solved).  The status is
 * OK only when every system converged.  nrhs is padded to a power of two
 * with zero systems internally. */
qcd_status qcd_solve_cg_multi(const qcd_gauge *g, qcd_spinor *const *x, const qcd_spinor *const *b, int nrhs,
                              const qcd_solver_params *params, qcd_solver_stats *stats, void *stream);

/* n (1..32) systems that share the gauge field but have their own hopping
 * parameter, twisted mass and tolerance -- params[k] for system k -- solved
 * by one batched CG, as qcd_solve_cg_multi (batching over sources and kappa
 * values).  All kappa/mu-dependent epilogue coefficients are read per
 * right-hand side from a device table.  params[k].maxiter, eo, normal,
 * inner_prec, inner_recon and reliable_delta must be the same for every k
 * (INVALID_ARG otherwise); systems that converge first stop changing while
 * the rest continue, and a reliable update of one is a reliable update of
 * all.  Errors as for qcd_solve_cg_multi. */
qcd_status qcd_solve_cg_batch(const qcd_gauge *g, qcd_spinor *const *x, const qcd_spinor *const *b, int n,
                              const qcd_solver_params *params, qcd_solver_stats *stats, void *stream);

/* n (1..32) independent even-odd FP64 CG solves -- each with its own gauge
 * field, lattice volume, hopping parameter, twisted mass and tolerance --
 * advanced together by ONE persistent cooperative kernel launch (source
 * preparation, CG, FP64 true-residual check, odd-site reconstruction and the
 * full-system residual, separated by grid-wide barriers instead of kernel
 * launches).  Meant for small lattices, where one solve cannot fill the GPU:
 * the paper's finite-temperature studies are many independent runs over
 * couplings and volumes (Sec. 1) within device memory (Sec. 2).
 * gauges[k]: F64 field; x[k], b[k]: FULL F64 spinors on one lattice with the
 * gauge field's extents -- its own lattice or another handle (a context
 * lattice, which then holds the scratch, so that calls on different context
 * lattices may run concurrently on the same gauge field); distinct x;
 * params[k].eo = 1, normal = 0, inner_prec = F64, one maxiter for all.
 * Blocks are shared out in proportion to the site counts, so each result is
 * bitwise the same alone and in any batch.  max_blocks (0: as many as fit
 * the GPU at once, else at least n) caps the grid, so a caller that shares
 * the GPU with other work does not wait for all of it to be free: a
 * cooperative launch starts only once every block is resident.
 * wait_cycles bounds every barrier wait (0: about two seconds); when a wait
 * runs out the call returns QCD_ERR_TIMEOUT and the context stays usable.  The systems' lattice
 * handles hold the scratch fields, so calls that share a lattice must not
 * overlap on the device.  Synchronous (returns after the stats are final);
 * errors as for qcd_solve_cg, per system in stats. */
qcd_status qcd_solve_cg_many(int n, const qcd_gauge *const *gauges, qcd_spinor *const *x, const qcd_spinor *const *b,
                             const qcd_solver_params *params, qcd_solver_stats *stats, long long wait_cycles,
                             int max_blocks, void *stream);

/* ---------------------------------------------------- time-slab split
 * The paper splits the lattice in the time direction across devices
 * (Sec. 7).  A rank holding Lt_loc consecutive time slices (Lt_loc even, so
 * even-odd parities agree with the global ones up to one swap) works on an
 * EXTENDED lattice of Lt_loc + 2 slices created with t_bc = +1: slices
 * 1 .. Lt_loc are its own, slices 0 and Lt_loc + 1 are halos.  Its gauge
 * field holds the rank's links on the own slices and identity links on the
 * halo slices.  Before each hopping-term application on a half field `in`:
 *   qcd_face_pack(TO_PREV): h = psi_up - S psi_dn of own slice 1 (S = +1 for
 *     D, -1 for D^dagger), for the previous rank's forward t hops;
 *   qcd_face_pack(TO_NEXT): u = U_t(x)^dagger (psi_up + S psi_dn) of the last
 *     own slice, for the next rank's backward t hops;
 *   `sign` multiplies the face: t_bc where the face crosses the global time
 *   boundary (the previous rank of rank 0 is the last rank), else 1;
 *   the faces are exchanged by the caller into the receiver's own device
 *   buffers, and qcd_face_unpack(FROM_NEXT / FROM_PREV) writes them into
 *   the halo slices (upper spins = face, lower spins = 0);
 *   qcd_apply_dslash on the extended lattice then gives D_eo (or D_eo^dag)
 *   on the own slices.  Faces are 6 complex per site of one parity in one
 *   time slice: face_dev holds 6 * (Lx Ly Lz / 2) double2, component-major.
 * F64 fields and gauge only; INVALID_ARG for other fields or a lattice that
 * is not an extended slab (t_bc = +1, >= 4 slices).  Asynchronous on
 * `stream`. */
#define QCD_FACE_TO_PREV 0
#define QCD_FACE_TO_NEXT 1
#define QCD_FACE_FROM_PREV 2
#define QCD_FACE_FROM_NEXT 3
qcd_status qcd_face_pack(const qcd_gauge *g, const qcd_spinor *in, int face, int dagger, double sign, double *face_dev,
                         void *stream);
qcd_status qcd_face_unpack(qcd_spinor *out, int face, const double *face_dev, void *stream);

/* ----------------------------------------------------------------- server */

/* A solve server: independent even-odd CG solves of different volumes and
 * parameters, admitted as slots and device memory free up and run
 * concurrently, one CUDA stream per slot.  The paper notes that
 * finite-temperature studies are a naturally parallel set of independent
 * simulations over couplings and volumes (Sec. 1), bounded by device memory
 * (Sec. 2).  Gauge fields stay resident (registered once, shared read-only);
 * each slot keeps per-volume solver contexts; a request is admitted in
 * arrival order when a slot is free and its context fits memory_budget
 * (idle contexts of that slot are released to make room).  A solve's result
 * does not depend on what else runs (same kernels, launch shapes and
 * fixed-order reductions).  All entry points are thread-safe. */
typedef struct qcd_server qcd_server;
typedef struct {
    int slots;             /* concurrent solves (1..64) */
    size_t memory_budget;  /* device bytes the solver contexts may use */
    int batch_small_sites; /* 0 (default): off; else requests on lattices of at
                              most this many sites that are queued together
                              (up to 16, same maxiter) run as one
                              qcd_solve_cg_many launch (FP64 CG to each
                              request's tolerance).  A cooperative launch
                              waits for, then holds, the SMs other slots'
                              solves want, so it pays only when small
                              requests dominate the stream. */
} qcd_server_config;
typedef struct {
    int gauge_id;          /* from qcd_server_add_gauge */
    double kappa, mu, tol;
    int maxiter;
    qcd_prec inner_prec;   /* as qcd_solver_params (even-odd solve of M x = b) */
    qcd_recon inner_recon;
    double reliable_delta;  /* as qcd_solver_params (0: by inner precision) */
    const double *b_host;  /* full source, host layout; valid until the request completes */
    double *x_host;        /* full solution, written before completion */
} qcd_request;
typedef struct {
    long long id;
    int status;            /* the solve's qcd_status */
    int slot;
    qcd_solver_stats stats;
    double t_submit, t_start, t_end; /* seconds since qcd_server_create */
} qcd_request_result;
/* Errors: INVALID_ARG; CUDA (stream creation). */
qcd_status qcd_server_create(const qcd_server_config *cfg, qcd_server **out);
/* Register a resident F64 gauge field (the caller keeps it alive and
 * unchanged while the server runs; prepare the inner precisions with
 * qcd_gauge_prepare first). */
qcd_status qcd_server_add_gauge(qcd_server *sv, const qcd_gauge *g, int *gauge_id);
/* Queue a request; returns at once with its id.  OOM if the request alone
 * needs more than the whole budget. */
qcd_status qcd_server_submit(qcd_server *sv, const qcd_request *req, long long *request_id);
/* Block until the request completes; fills `out` and forgets the request. */
qcd_status qcd_server_wait(qcd_server *sv, long long request_id, qcd_request_result *out);
/* Bytes reserved by solver contexts, queued and running request counts. */
qcd_status qcd_server_info(qcd_server *sv, size_t *used_bytes, int *queued, int *running);
/* Stop the server: queued requests end with QCD_ERR_CANCELLED (a thread
 * blocked in qcd_server_wait on one returns with that status), running
 * requests finish, and the call returns once no thread is inside
 * qcd_server_wait; then the contexts are freed.  Requests not yet waited for
 * are dropped.  No call may use the handle after this one has begun. */
void qcd_server_destroy(qcd_server *sv);

/* ------------------------------------------------------------ measurement */

/* The paper's kernel classes carry the number of FLOPs each kernel performs
 * so that performance can be reported (Sec. 4), and it rates the Dslash by
 * its achieved memory bandwidth (Sec. 1, Sec. 6).  Between
 * qcd_profile_begin and qcd_profile_end every hopping-kernel launch is
 * bracketed by CUDA events on its own stream, and its algorithmic traffic
 * and flops are recorded:
 *   bytes = sites * (8 links + 1 input spinor + 1 output spinor
 *                    [+ 1 spinor y of the fused epilogue]),
 *           in the storage precision (links at 18 or 12 reals; FP16
 *           spinors include their 4-byte scale);
 *   flops = 1320 per output site (projection, two SU(3) products and the
 *           accumulation of 8 hops; the rebuilt third link row and the
 *           epilogue are not counted).
 * Entries are indexed by qcd_prec.  One profiling window at a time, from
 * one host thread.  qcd_profile_end waits for the recorded events. */
typedef struct {
    long long launches;
    double ms;     /* summed device time of the launches */
    double bytes;  /* summed algorithmic bytes */
    double flops;  /* summed algorithmic flops */
    double sites;  /* summed output sites */
} qcd_profile_entry;
typedef struct {
    qcd_profile_entry prec[5];
} qcd_profile;
qcd_status qcd_profile_begin(void);
qcd_status qcd_profile_end(qcd_profile *out);
/* Number of CUDA kernels this library has launched since it was loaded. */
unsigned long long qcd_kernel_launches(void);

/* Launch shape of the FP64 reconstruct-18 hopping kernel (one right-hand
 * side): 0 (default) lets the autotuner choose between one thread per
 * output site and eight (one hop each, for small lattices); 1 or 8 forces
 * that choice for later launches (tests and benchmarks of either kernel).
 * The paper compiles kernels per configuration (Sec. 4); here both are
 * compiled and one is picked per lattice.  INVALID_ARG for other values. */
qcd_status qcd_set_hop_threads(int threads_per_site);

/* Host-side failure injection for tests of the error paths (no device
 * fault is involved): the next `count` calls of kind `what` fail with
 * QCD_ERR_OOM before touching the device.  QCD_INJECT_SPINOR_CREATE:
 * qcd_spinor_create.  count = 0 clears.  The paper has no counterpart (its
 * Sec. 5 asks that every part of the code be testable on its own). */
#define QCD_INJECT_SPINOR_CREATE 1
qcd_status qcd_debug_inject(int what, int count);

#ifdef __cplusplus
}
#endif

#endif /* QCD_H */
