// C ABI of libqcd: handles, host<->device transfer, operator application.
// Declarations and argument conventions are in include/qcd.h.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "qcd_handles.h"

namespace qcd {

static thread_local char g_err[512] = "";
// set by lattice_create_on for the duration of one qcd_lattice_create call
static thread_local cudaStream_t g_create_stream = nullptr;
static std::atomic<unsigned long long> g_launches{0};

std::shared_mutex &device_mutex()
{
    static std::shared_mutex m;
    return m;
}

void note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

// ---- host-side failure injection (qcd_debug_inject): the next `count`
// calls of the chosen kind fail as if their allocation had failed
static std::atomic<int> g_inject[2] = {};

static bool take_injected_failure(int what)
{
    std::atomic<int> &n = g_inject[what];
    int v = n.load();
    while (v > 0)
        if (n.compare_exchange_weak(v, v - 1)) return true;
    return false;
}

// ---- hopping-kernel profiling (qcd_profile_begin / qcd_profile_end)
struct ProfRec {
    cudaEvent_t e0, e1;
    int prec;
    double bytes, flops, sites;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_event_pool;

bool profiling_active() { return g_prof_on; }

static cudaEvent_t pool_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static double spinor_site_bytes(int prec)
{
    switch (prec) {
    case QCD_PREC_F64:
    case QCD_PREC_DF64: return 192;
    case QCD_PREC_F32: return 96;
    case QCD_PREC_F16: return 52;
    default: return 48;
    }
}
static double link_bytes(int prec, int recon)
{
    const double w = (prec == QCD_PREC_F64 || prec == QCD_PREC_DF64) ? 8 : prec == QCD_PREC_F32 ? 4 : 2;
    return w * recon;
}

qcd_status fail(qcd_status code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

qcd_status check_cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return QCD_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(QCD_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    if (e == cudaErrorInvalidValue) return fail(QCD_ERR_INVALID_ARG, "%s: unsupported format or argument", what);
    return fail(QCD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ----------------------------------------------------------------- sizes

int spinor_planes(int prec) { return (prec == QCD_PREC_F64 || prec == QCD_PREC_DF64) ? 12 : prec == QCD_PREC_F32 ? 6 : 3; }
size_t spinor_plane_elem_bytes(int) { return 16; }
size_t spinor_half_bytes(int prec, int stride) { return (size_t)spinor_planes(prec) * 16 * stride; }
size_t spinor_half_norm_bytes(int prec, int stride) { return prec == QCD_PREC_F16 ? (size_t)4 * stride : 0; }

int gauge_planes(int prec, int recon)
{
    if (prec == QCD_PREC_F64 || prec == QCD_PREC_DF64) return recon / 2;
    if (recon == 8) return prec == QCD_PREC_F32 ? 2 : 1;
    return recon == 18 ? 9 : 3;
}
size_t gauge_plane_elem_bytes(int prec, int recon)
{
    if (prec == QCD_PREC_F64 || prec == QCD_PREC_DF64 || recon == 8) return 16;
    if (prec == QCD_PREC_F32) return recon == 18 ? 8 : 16;
    return recon == 18 ? 4 : 8;
}
size_t gauge_bytes(int prec, int recon, int stride)
{
    return (size_t)8 * gauge_planes(prec, recon) * gauge_plane_elem_bytes(prec, recon) * stride;
}

static bool valid_prec(int p) { return p >= QCD_PREC_F64 && p <= QCD_PREC_DF64; }
static bool valid_recon(int r) { return r == 18 || r == 12 || r == 8; }

// Largest entry error a reconstruct-8 field may show against its FP64
// source before it is refused: 4 units of the 16-bit roundoff (the storage
// rounding itself is 0.5), 32 of FP32 (the FP32 rebuild costs ~7), and
// 1e-13 in FP64.  Links far from the identity exceed these, since the
// pivot assumes large diagonal entries.
static double recon8_tolerance(int prec)
{
    switch (prec) {
    case QCD_PREC_F64: return 1e-13;
    case QCD_PREC_F32: return 32.0 * 0x1p-24;
    case QCD_PREC_F16: return 4.0 * 0x1p-11;
    case QCD_PREC_BF16: return 4.0 * 0x1p-8;
    default: return 0.0;
    }
}

static const char *prec_name(int prec)
{
    static const char *n[] = {"F64", "F32", "F16", "BF16", "DF64"};
    return prec >= 0 && prec <= 4 ? n[prec] : "?";
}

// Validate a freshly written reconstruct-8 field (synchronises `s`).
static qcd_status check_recon8(const GaugeView &dst, int prec, const double2 *aos, const GaugeView &src, int sprec,
                               int srecon, const Geom &g, cudaStream_t s, const char *what)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return fail(QCD_ERR_INVALID_ARG, "%s: a reconstruct-8 copy is validated on the host; prepare it outside stream capture",
                    what);
    double err = 0.0;
    cudaError_t e = gauge_recon8_error(dst, prec, aos, src, sprec, srecon, g, s, &err);
    if (e != cudaSuccess) return check_cuda(e, what);
    const double tol = recon8_tolerance(prec);
    if (!(err <= tol))
        return fail(QCD_ERR_INVALID_ARG,
                    "%s: reconstruct-8 in %s misses these links by %.3g (limit %.3g): the pivoted 8-real form needs "
                    "links near the identity; use reconstruct-12",
                    what, prec_name(prec), err, tol);
    return QCD_OK;
}

// ----------------------------------------------------------------- memory

// Device memory of a lattice's buffers: stream-ordered on lat->alloc_stream
// when it is set (no device-wide synchronisation), else cudaMalloc/cudaFree.
static cudaError_t lat_alloc(const qcd_lattice *lat, void **p, size_t n)
{
    return lat && lat->alloc_stream ? cudaMallocAsync(p, n, lat->alloc_stream) : cudaMalloc(p, n);
}
static void lat_free(const qcd_lattice *lat, void *p)
{
    if (!p) return;
    if (lat && lat->alloc_stream)
        cudaFreeAsync(p, lat->alloc_stream);
    else
        cudaFree(p);
}
cudaError_t zero_now(void *p, size_t n);
static cudaError_t lat_zero(const qcd_lattice *lat, void *p, size_t n)
{
    return lat && lat->alloc_stream ? cudaMemsetAsync(p, 0, n, lat->alloc_stream) : zero_now(p, n);
}

// Pinned staging buffers (CG state mirror, coefficient table) of
// stream-ordered lattices are reused instead of freed: cudaFreeHost may
// synchronise the device.
static std::mutex g_pinned_mu;
static std::vector<std::pair<void *, void *>> g_pinned_pool;

static cudaError_t pinned_get(void **state, void **coef)
{
    {
        std::lock_guard<std::mutex> lk(g_pinned_mu);
        if (!g_pinned_pool.empty()) {
            *state = g_pinned_pool.back().first;
            *coef = g_pinned_pool.back().second;
            g_pinned_pool.pop_back();
            return cudaSuccess;
        }
    }
    cudaError_t e = cudaMallocHost(state, sizeof(CgState));
    if (e == cudaSuccess) e = cudaMallocHost(coef, kCoefHostDoubles * sizeof(double));
    return e;
}
static void pinned_put(void *state, void *coef)
{
    if (!state || !coef) {
        if (state) cudaFreeHost(state);
        if (coef) cudaFreeHost(coef);
        return;
    }
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    g_pinned_pool.emplace_back(state, coef);
}

// ----------------------------------------------------------------- views

void *workspace(const qcd_lattice *lat, const std::string &name, size_t bytes)
{
    auto it = lat->ws.find(name);
    if (it != lat->ws.end() && it->second.second >= bytes) return it->second.first;
    if (lat->alloc_stream) {
        // stream-ordered: only this lattice's own stream is waited for
        if (it != lat->ws.end()) {
            cudaStreamSynchronize(lat->alloc_stream);
            for (auto &kv : lat->graphs) {
                cudaGraphExecDestroy(kv.second.exec);
                cudaGraphDestroy(kv.second.graph);
            }
            lat->graphs.clear();
            lat_free(lat, it->second.first);
            lat->ws.erase(it);
        }
        void *p = nullptr;
        if (lat_alloc(lat, &p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        lat->ws[name] = {p, bytes};
        return p;
    }
    DeviceLock dl(device_mutex());
    if (it != lat->ws.end()) {
        // cached CG graphs may hold this buffer's address: drop them all
        cudaDeviceSynchronize();
        for (auto &kv : lat->graphs) {
            cudaGraphExecDestroy(kv.second.exec);
            cudaGraphDestroy(kv.second.graph);
        }
        lat->graphs.clear();
        cudaFree(it->second.first);
        lat->ws.erase(it);
    }
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    lat->ws[name] = {p, bytes};
    return p;
}

FieldView view_half(const qcd_spinor *s, int half)
{
    FieldView f;
    f.nh = 1;
    f.h = s->lat->h;
    f.prec = s->prec;
    f.rhs_log2 = 0;
    f.hv[0].data = static_cast<char *>(s->data) + half * s->half_data_bytes;
    f.hv[0].norm = s->norm ? reinterpret_cast<float *>(reinterpret_cast<char *>(s->norm) + half * s->half_norm_bytes)
                           : nullptr;
    f.hv[0].stride = s->lat->stride;
    f.hv[1] = f.hv[0];
    return f;
}

FieldView view_of(const qcd_spinor *s)
{
    FieldView f = view_half(s, 0);
    if (s->parity == QCD_PARITY_FULL) {
        f.nh = 2;
        f.hv[1] = view_half(s, 1).hv[0];
    }
    return f;
}

FieldView ws_field(const qcd_lattice *lat, const std::string &name, int nh, int prec, int rhs_log2)
{
    // fits an int: lattice creation demands h * Lmax < 2^32 with Lmax >=
    // (2h)^(1/4), so h < 2^25.4 and h * kMaxRhs * 2 parities < 2^30.4
    const int ne = lat->h << rhs_log2;
    const int stride = rhs_log2 == 0 ? lat->stride : (ne + 63) / 64 * 64;
    const size_t db = spinor_half_bytes(prec, stride), nb = spinor_half_norm_bytes(prec, stride);
    char *base = static_cast<char *>(
        workspace(lat, name + "/p" + std::to_string(prec) + "/n" + std::to_string(rhs_log2), nh * (db + nb)));
    FieldView f;
    f.nh = nh;
    f.h = ne;
    f.prec = prec;
    f.rhs_log2 = rhs_log2;
    for (int k = 0; k < 2; ++k) {
        const int kk = k < nh ? k : 0;
        f.hv[k].data = base ? base + kk * db : nullptr;
        f.hv[k].norm = (base && nb) ? reinterpret_cast<float *>(base + nh * db + kk * nb) : nullptr;
        f.hv[k].stride = stride;
    }
    return f;
}

Reduction reduction_of(const qcd_lattice *lat) { return Reduction{lat->red_partials, lat->red_counter, lat->red_cap}; }

// Zero a new device buffer before any stream may use it.  A plain memset
// runs on the legacy default stream, which non-blocking streams (a server
// slot's, a user's) do not wait for: finished here, it cannot land after
// the first kernels that read or fill the buffer.
cudaError_t zero_now(void *p, size_t n)
{
    cudaError_t e = cudaMemsetAsync(p, 0, n, cudaStreamLegacy);
    return e == cudaSuccess ? cudaStreamSynchronize(cudaStreamLegacy) : e;
}

GaugeView gauge_view(const qcd_gauge *g, int prec, int recon, cudaStream_t s, qcd_status *st)
{
    *st = QCD_OK;
    const int stride = g->lat->stride;
    if (prec == g->prec && recon == g->recon) return GaugeView{g->data, stride};
    const int key = prec * 100 + recon;
    auto *gm = const_cast<qcd_gauge *>(g);
    static std::mutex derived_mu;  // concurrent solves may share one gauge field
    std::lock_guard<std::mutex> lk(derived_mu);
    auto it = gm->derived.find(key);
    if (it != gm->derived.end()) return GaugeView{it->second.first, stride};
    // The copy is converted on `s` and then published to every stream, so
    // the conversion must be complete first: it is built outside stream
    // capture and the stream is synchronised before the pointer is stored.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        *st = fail(QCD_ERR_INVALID_ARG, "gauge copy: a copy in a new precision is built outside stream capture "
                                        "(call qcd_gauge_prepare first)");
        return GaugeView{nullptr, stride};
    }
    const size_t bytes = gauge_bytes(prec, recon, stride);
    void *p = nullptr;
    DeviceLock dl(device_mutex());
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *st = fail(QCD_ERR_OOM, "gauge copy: cudaMalloc(%zu) failed", bytes);
        return GaugeView{nullptr, stride};
    }
    const GaugeView dst{p, stride}, src{g->data, stride};
    cudaError_t e = launch_gauge_convert(dst, prec, recon, src, g->prec, g->recon, g->lat->geom, s);
    if (e != cudaSuccess) {
        cudaFree(p);
        *st = check_cuda(e, "gauge copy");
        return GaugeView{nullptr, stride};
    }
    if (recon == 8) {
        *st = check_recon8(dst, prec, nullptr, src, g->prec, g->recon, g->lat->geom, s, "gauge copy");
        if (*st != QCD_OK) {
            cudaFree(p);
            return GaugeView{nullptr, stride};
        }
    }
    e = cudaStreamSynchronize(s);  // other streams may use the copy as soon as it is stored
    if (e != cudaSuccess) {
        cudaFree(p);
        *st = check_cuda(e, "gauge copy");
        return GaugeView{nullptr, stride};
    }
    gm->derived[key] = {p, bytes};
    return dst;
}

// ----------------------------------------------------------------- hop

Coef coef_twist(double b)
{
    Coef c;
    c.c[0][0] = 1.0;
    c.c[0][1] = b;
    c.c[1][0] = 1.0;
    c.c[1][1] = -b;
    return c;
}
Coef coef_twist_inv(double b)
{
    const double n = 1.0 / (1.0 + b * b);
    Coef c;
    c.c[0][0] = n;
    c.c[0][1] = -b * n;
    c.c[1][0] = n;
    c.c[1][1] = b * n;
    return c;
}
Coef coef_scale(Coef c, double s)
{
    for (auto &k : c.c)
        for (double &v : k) v *= s;
    return c;
}
Coef coef_real(double s)
{
    Coef c;
    c.c[0][0] = c.c[1][0] = s;
    c.c[0][1] = c.c[1][1] = 0.0;
    return c;
}

cudaError_t launch_dslash_f64(int recon, const DslashLaunch &a, cudaStream_t s);
cudaError_t launch_dslash_f32(int recon, const DslashLaunch &a, cudaStream_t s);
cudaError_t launch_dslash_f16(int recon, const DslashLaunch &a, cudaStream_t s);
cudaError_t launch_dslash_bf16(int recon, const DslashLaunch &a, cudaStream_t s);
cudaError_t launch_dslash_df64_d0(int recon, const DslashLaunch &a, cudaStream_t s);
cudaError_t launch_dslash_df64_d1(int recon, const DslashLaunch &a, cudaStream_t s);

cudaError_t launch_dslash(int prec, int recon, const DslashLaunch &a, cudaStream_t s)
{
    switch (prec) {
    case QCD_PREC_F64: return launch_dslash_f64(recon, a, s);
    case QCD_PREC_F32: return launch_dslash_f32(recon, a, s);
    case QCD_PREC_F16: return launch_dslash_f16(recon, a, s);
    case QCD_PREC_BF16: return launch_dslash_bf16(recon, a, s);
    case QCD_PREC_DF64: return a.dagger ? launch_dslash_df64_d1(recon, a, s) : launch_dslash_df64_d0(recon, a, s);
    default: return cudaErrorInvalidValue;
    }
}

// ---- autotuner of the hopping-kernel block size
//
// The paper compiles its kernels for the lattice at hand and keeps the
// compiled binaries for later runs (Sec. 4).  Here the kernels are compiled
// ahead of time; what depends on the lattice is the launch shape.  The
// first launch of a (precision, recon, batch, parity layout, extents)
// configuration outside stream capture times the FP32/16-bit kernel with 64,
// 128 and 256 threads per block (CUDA events, three launches each on
// scratch fields) and keeps the fastest.  FP64 reconstruct-18 launches with
// one right-hand side choose between one thread per site (64-thread blocks)
// and the eight-lane kernel (one hop per thread, 128-thread blocks), the
// latter winning on small lattices; a choice is stored as
// tpb | (threads per site << 16).  With QCD_TUNE_CACHE=<file> the choices
// are read from and appended to that file, so later processes skip the
// timing.
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune;
static bool g_tune_loaded = false;
static std::atomic<int> g_force_tps{0};  // qcd_set_hop_threads: 0 autotuned, 1 or 8 forced

static bool valid_tune(int v)
{
    const int tpb = v & 0xffff, tps = v >> 16;
    return (tpb == 64 || tpb == 128 || tpb == 256) && (tps == 0 || (tps == 8 && tpb == 128));
}

static void tune_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("QCD_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char key[256];
    int v;
    while (fscanf(f, "%255s %d", key, &v) == 2)
        if (valid_tune(v)) g_tune[key] = v;
    fclose(f);
}

static void tune_store(const std::string &key, int v)
{
    g_tune[key] = v;
    const char *path = getenv("QCD_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d\n", key.c_str(), v);
    fclose(f);
}

static std::string tune_key(const qcd_lattice *lat, int prec, int recon, int L, bool both)
{
    char k[160];
    snprintf(k, sizeof(k), "dslash:p%d:r%d:n%d:b%d:%dx%dx%dx%d", prec, recon, L, both ? 1 : 0, lat->dims[0], lat->dims[1],
             lat->dims[2], lat->dims[3]);
    return k;
}

constexpr int kLanes8 = 128 | (8 << 16);

// Batched fields: blocks run in t-major order (DslashLaunch::tmap) when they
// tile the time slices; the one-thread kernels' block size is 64 for FP64
// and DF64, else tpb.  Measured on a 16-rhs FP32 launch at 32^3x8 in site
// order: 768 MB of DRAM traffic against 453 MB algorithmic, since the input
// (201 MB) exceeds L2 and the y/z/t neighbours were read again from DRAM.
static int tmap_of(const qcd_lattice *lat, int prec, int rhs_log2, int tpb, int split)
{
    const int bs = (prec == QCD_PREC_F64 || prec == QCD_PREC_DF64) ? 64 : tpb;
    const long long per_slice = (long long)lat->geom.st << rhs_log2;
    return (rhs_log2 > 0 && split == 1 && per_slice % bs == 0) ? (int)(per_slice / bs) : 0;
}

int tuned_tpb(const qcd_lattice *lat, const GaugeView &U, int prec, int recon, int L, bool both, cudaStream_t s)
{
    const bool lanes8_ok = prec == QCD_PREC_F64 && recon == 18 && L == 0;
    if ((prec == QCD_PREC_F64 && !lanes8_ok) || prec == QCD_PREC_DF64) return 64;
    const int force = g_force_tps.load();
    if (lanes8_ok && force == 8) return kLanes8;
    if (lanes8_ok && force == 1) return 64;
    const std::string key = tune_key(lat, prec, recon, L, both);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return it->second;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const int fallback = lanes8_ok ? 64 : 128;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return fallback;
    const FieldView ti = ws_field(lat, "tune_in", both ? 2 : 1, prec, L);
    const FieldView to = ws_field(lat, "tune_out", both ? 2 : 1, prec, L);
    if (!ti.hv[0].data || !to.hv[0].data || launch_zero(ti, s) != cudaSuccess) return fallback;
    DslashLaunch a;
    memset(&a, 0, sizeof(a));
    a.g = lat->geom;
    a.both = both ? 1 : 0;
    a.rhs_log2 = L;
    a.U = U;
    for (int p = 0; p < 2; ++p) {
        a.out[p] = to.hv[both ? p : 0];
        a.in[p] = ti.hv[both ? 1 - p : 0];
    }
    a.epi = EPI_PLAIN;
    a.state = lat->state;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = fallback;
    float best_ms = 1e30f;
    const std::vector<int> cand = lanes8_ok ? std::vector<int>{64, kLanes8} : std::vector<int>{128, 64, 256};
    for (int v : cand) {
        a.tpb = v & 0xffff;
        a.split = (v >> 16) == 8 ? 8 : 1;
        a.tmap = tmap_of(lat, prec, L, a.tpb, a.split);
        bool ok = launch_dslash(prec, recon, a, s) == cudaSuccess;  // warm-up
        float ms_min = 1e30f;
        for (int r = 0; r < 3 && ok; ++r) {
            cudaEventRecord(e0, s);
            ok = launch_dslash(prec, recon, a, s) == cudaSuccess;
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                ms_min = ms < ms_min ? ms : ms_min;
        }
        note_launches(4);
        if (ok && ms_min < best_ms) {
            best_ms = ms_min;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_store(key, best);
    return best;
}

cudaError_t hop(const qcd_lattice *lat, const GaugeView &U, int recon, const HopArgs &h, cudaStream_t s)
{
    DslashLaunch a;
    memset(&a, 0, sizeof(a));
    a.g = lat->geom;
    a.out_parity = h.out_parity;
    a.both = h.both ? 1 : 0;
    a.rhs_log2 = h.out->rhs_log2;
    a.dagger = h.dagger;
    a.U = U;
    if (h.both) {
        for (int p = 0; p < 2; ++p) {
            a.out[p] = h.out->hv[p];
            a.in[p] = h.in->hv[1 - p];
            if (h.y) a.y[p] = h.y->hv[p];
        }
    } else {
        const int p = h.out_parity;
        a.out[p] = h.out->hv[0];
        a.in[p] = h.in->hv[0];
        if (h.y) a.y[p] = h.y->hv[0];
    }
    memcpy(a.cy, h.cy.c, sizeof(a.cy));
    memcpy(a.cd, h.cd.c, sizeof(a.cd));
    for (int k = 0; k < 4; ++k) {
        a.cyf[k >> 1][k & 1] = (float)a.cy[k >> 1][k & 1];
        a.cdf[k >> 1][k & 1] = (float)a.cd[k >> 1][k & 1];
    }
    if (h.coef && !h.coef_f) return cudaErrorInvalidValue;
    a.coef = h.coef;
    a.coef_f = h.coef_f;
    a.coef_stride = h.coef_stride;
    if (h.plain)
        a.epi = EPI_PLAIN;
    else if (!h.y)
        a.epi = EPI_CPLX_D;  // out = cd .* D in (real coefficients are the im = 0 case)
    else
        a.epi = h.twisted ? EPI_CPLX_YD : EPI_REAL_YD;
    const int cfg = tuned_tpb(lat, U, h.out->prec, recon, h.out->rhs_log2, h.both, s);
    a.tpb = cfg & 0xffff;
    a.split = (cfg >> 16) == 8 ? 8 : 1;
    a.tmap = tmap_of(lat, h.out->prec, h.out->rhs_log2, a.tpb, a.split);
    a.reduce = h.reduce;
    a.red = h.red ? *h.red : reduction_of(lat);
    if (h.reduce) {
        const int tpb = a.tpb;
        const size_t blocks =
            (size_t)((((size_t)lat->h << h.out->rhs_log2) * a.split + tpb - 1) / tpb) * (h.both ? 2 : 1);
        if (!reduction_fits(a.red, 1, h.out->rhs_log2, blocks)) return cudaErrorInvalidValue;
    }
    a.fin = h.fin;
    a.state = lat->state;
    a.red_out = lat->red_out;
    a.check_status = h.check_status;
    a.run_status = h.run_status;
    const bool prof = g_prof_on;
    if (!prof) {
        note_launches();
        return launch_dslash(h.out->prec, recon, a, s);
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfRec r;
    r.e0 = pool_event();
    r.e1 = pool_event();
    r.prec = h.out->prec;
    r.sites = (double)(lat->h << h.out->rhs_log2) * (h.both ? 2 : 1);  // site x rhs elements
    r.bytes = (double)lat->h * (h.both ? 2 : 1) * 8 * link_bytes(h.out->prec, recon) +
              r.sites * (h.y ? 3 : 2) * spinor_site_bytes(h.out->prec);
    r.flops = r.sites * 1320.0;
    cudaEventRecord(r.e0, s);
    note_launches();
    cudaError_t e = launch_dslash(h.out->prec, recon, a, s);
    cudaEventRecord(r.e1, s);
    g_prof.push_back(r);
    return e;
}

}  // namespace qcd

using namespace qcd;

qcd_status qcd::lattice_create_on(const int dims[4], int t_bc, cudaStream_t s, qcd_lattice **out)
{
    g_create_stream = s;
    const qcd_status st = qcd_lattice_create(dims, t_bc, out);
    g_create_stream = nullptr;
    return st;
}

// =================================================================== C ABI

extern "C" {

const char *qcd_status_string(qcd_status s)
{
    switch (s) {
    case QCD_OK: return "QCD_OK";
    case QCD_ERR_INVALID_ARG: return "QCD_ERR_INVALID_ARG";
    case QCD_ERR_OOM: return "QCD_ERR_OOM";
    case QCD_ERR_CUDA: return "QCD_ERR_CUDA";
    case QCD_ERR_NOT_CONVERGED: return "QCD_ERR_NOT_CONVERGED";
    case QCD_ERR_BREAKDOWN: return "QCD_ERR_BREAKDOWN";
    case QCD_ERR_TIMEOUT: return "QCD_ERR_TIMEOUT";
    case QCD_ERR_CANCELLED: return "QCD_ERR_CANCELLED";
    default: return "QCD_ERR_UNKNOWN";
    }
}

const char *qcd_last_error(void) { return g_err; }

const char *qcd_version(void) { return "libqcd 0.1 (sm_103a)"; }

unsigned long long qcd_kernel_launches(void) { return g_launches.load(); }

qcd_status qcd_set_hop_threads(int threads_per_site)
{
    if (threads_per_site != 0 && threads_per_site != 1 && threads_per_site != 8)
        return fail(QCD_ERR_INVALID_ARG, "set_hop_threads: %d is not 0, 1 or 8", threads_per_site);
    g_force_tps.store(threads_per_site);
    return QCD_OK;
}

qcd_status qcd_debug_inject(int what, int count)
{
    if (what != QCD_INJECT_SPINOR_CREATE || count < 0)
        return fail(QCD_ERR_INVALID_ARG, "debug_inject: unknown kind %d or negative count", what);
    g_inject[what].store(count);
    return QCD_OK;
}

qcd_status qcd_profile_begin(void)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_on) return fail(QCD_ERR_INVALID_ARG, "profile_begin: a profiling window is already open");
    g_prof.clear();
    g_prof_on = true;
    return QCD_OK;
}

qcd_status qcd_profile_end(qcd_profile *out)
{
    if (!out) return fail(QCD_ERR_INVALID_ARG, "profile_end: NULL argument");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return fail(QCD_ERR_INVALID_ARG, "profile_end: no profiling window is open");
    g_prof_on = false;
    memset(out, 0, sizeof(*out));
    qcd_status st = QCD_OK;
    for (const ProfRec &r : g_prof) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.e0, r.e1);
        if (e != cudaSuccess && st == QCD_OK) st = check_cuda(e, "profile_end");
        qcd_profile_entry &p = out->prec[r.prec];
        p.launches += 1;
        p.ms += ms;
        p.bytes += r.bytes;
        p.flops += r.flops;
        p.sites += r.sites;
        g_event_pool.push_back(r.e0);
        g_event_pool.push_back(r.e1);
    }
    g_prof.clear();
    return st;
}

qcd_status qcd_stream_sync(void *stream)
{
    return check_cuda(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "stream_sync");
}

qcd_status qcd_lattice_create(const int dims[4], int t_bc, qcd_lattice **out)
{
    if (!dims || !out) return fail(QCD_ERR_INVALID_ARG, "lattice_create: NULL argument");
    *out = nullptr;
    if (t_bc != 1 && t_bc != -1) return fail(QCD_ERR_INVALID_ARG, "lattice_create: t_bc must be +1 or -1");
    uint64_t V = 1;
    int lmax = 0;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2 || dims[mu] % 2) return fail(QCD_ERR_INVALID_ARG, "lattice_create: dims[%d] = %d must be even and >= 2", mu, dims[mu]);
        V *= (uint64_t)dims[mu];
        lmax = dims[mu] > lmax ? dims[mu] : lmax;
    }
    const uint64_t h = V / 2;
    // 32-bit site indices and the exactness bound of FastDiv (n * d < 2^32)
    if (V >= (1ull << 31) || h * (uint64_t)lmax >= (1ull << 32))
        return fail(QCD_ERR_INVALID_ARG, "lattice_create: volume too large");
    qcd_lattice *lat = new (std::nothrow) qcd_lattice();
    if (!lat) return fail(QCD_ERR_OOM, "lattice_create: host allocation");
    lat->alloc_stream = g_create_stream;
    DeviceLock dl(device_mutex(), std::defer_lock);
    if (!lat->alloc_stream) dl.lock();
    memcpy(lat->dims, dims, sizeof(lat->dims));
    lat->t_bc = t_bc;
    cudaGetDevice(&lat->device);
    Geom &g = lat->geom;
    for (int mu = 0; mu < 4; ++mu) g.L[mu] = dims[mu];
    g.Lxh = dims[0] / 2;
    g.h = (int)h;
    g.sy = g.Lxh;
    g.sz = g.Lxh * dims[1];
    g.st = g.Lxh * dims[1] * dims[2];
    g.dx = make_fastdiv(g.Lxh);
    g.dy = make_fastdiv(dims[1]);
    g.dz = make_fastdiv(dims[2]);
    g.tbc = (double)t_bc;
    lat->h = (int)h;
    lat->stride = (int)((h + 63) / 64 * 64);
    // partials of the largest grid: 128-thread blocks over eight work items
    // per site of all V sites (the eight-lane FP64 kernel), two values each
    const size_t bmax = ((size_t)V + 15) / 16;
    lat->red_cap = std::max(red_partials_needed(2, bmax), red_partials_needed(1, bmax));
    // tickets: one per group of the largest grid that shares them (64-thread
    // blocks over a batch of kMaxRhs full fields), and the final one
    const size_t counter_bytes = ((4 * (1 + (size_t)red_group_size((unsigned)(V * kMaxRhs / 64 + 1), 1)) + 255) / 256) * 256;
    cudaError_t e = lat_alloc(lat, (void **)&lat->red_partials, lat->red_cap * sizeof(double));
    if (e == cudaSuccess) e = lat_alloc(lat, (void **)&lat->red_counter, counter_bytes);
    if (e == cudaSuccess) e = lat_alloc(lat, (void **)&lat->red_out, 8 * sizeof(double));
    if (e == cudaSuccess) e = lat_alloc(lat, (void **)&lat->red_out_big, 2 * kMaxRhs * sizeof(double));
    if (e == cudaSuccess) e = lat_alloc(lat, (void **)&lat->state, sizeof(CgState));
    if (lat->alloc_stream) {
        if (e == cudaSuccess) e = pinned_get((void **)&lat->state_host, (void **)&lat->coef_host);
    } else {
        if (e == cudaSuccess) e = cudaMallocHost(&lat->state_host, sizeof(CgState));
        if (e == cudaSuccess) e = cudaMallocHost(&lat->coef_host, kCoefHostDoubles * sizeof(double));
    }
    if (e == cudaSuccess) e = lat_zero(lat, lat->red_counter, counter_bytes);
    if (e == cudaSuccess) e = lat_zero(lat, lat->state, sizeof(CgState));
    if (e != cudaSuccess) {
        qcd_status st = check_cuda(e, "lattice_create");
        if (dl.owns_lock()) dl.unlock();
        qcd_lattice_destroy(lat);
        return st;
    }
    *out = lat;
    return QCD_OK;
}

static void lattice_free(qcd_lattice *lat)
{
    if (lat->alloc_stream) {
        // stream-ordered: wait for this lattice's own stream only (its graphs
        // and staging must be idle), then free in stream order
        cudaStreamSynchronize(lat->alloc_stream);
        for (auto &kv : lat->graphs) {
            cudaGraphExecDestroy(kv.second.exec);
            cudaGraphDestroy(kv.second.graph);
        }
        for (void *p : {(void *)lat->red_partials, (void *)lat->red_counter, (void *)lat->red_out,
                        (void *)lat->red_out_big, (void *)lat->state})
            lat_free(lat, p);
        for (auto &kv : lat->ws) lat_free(lat, kv.second.first);
        pinned_put(lat->state_host, lat->coef_host);
        if (lat->capture_stream) cudaStreamDestroy(lat->capture_stream);
        delete lat;
        return;
    }
    DeviceLock dl(device_mutex());
    cudaDeviceSynchronize();
    cudaFree(lat->red_partials);
    cudaFree(lat->red_counter);
    cudaFree(lat->red_out);
    cudaFree(lat->red_out_big);
    cudaFree(lat->state);
    if (lat->state_host) cudaFreeHost(lat->state_host);
    if (lat->coef_host) cudaFreeHost(lat->coef_host);
    for (auto &kv : lat->ws) cudaFree(kv.second.first);
    for (auto &kv : lat->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
    }
    if (lat->capture_stream) cudaStreamDestroy(lat->capture_stream);
    delete lat;
}

static void lat_ref(const qcd_lattice *lat) { lat->refs.fetch_add(1); }

static void lat_unref(const qcd_lattice *lat)
{
    if (lat->refs.fetch_sub(1) == 1) lattice_free(const_cast<qcd_lattice *>(lat));
}

void qcd_lattice_destroy(qcd_lattice *lat)
{
    if (lat) lat_unref(lat);
}

qcd_status qcd_gauge_create(const qcd_lattice *lat, qcd_prec prec, qcd_recon recon, qcd_gauge **out)
{
    if (!lat || !out) return fail(QCD_ERR_INVALID_ARG, "gauge_create: NULL argument");
    *out = nullptr;
    if (!valid_prec(prec) || !valid_recon(recon)) return fail(QCD_ERR_INVALID_ARG, "gauge_create: bad prec/recon");
    qcd_gauge *g = new (std::nothrow) qcd_gauge();
    if (!g) return fail(QCD_ERR_OOM, "gauge_create: host allocation");
    g->lat = lat;
    g->prec = prec;
    g->recon = recon;
    g->bytes = gauge_bytes(prec, recon, lat->stride);
    DeviceLock dl(device_mutex());
    if (cudaMalloc(&g->data, g->bytes) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return fail(QCD_ERR_OOM, "gauge_create: cudaMalloc(%zu) failed", gauge_bytes(prec, recon, lat->stride));
    }
    if (zero_now(g->data, g->bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(g->data);
        delete g;
        return fail(QCD_ERR_CUDA, "gauge_create: zeroing the field failed");
    }
    lat_ref(lat);
    *out = g;
    return QCD_OK;
}

static void drop_derived(qcd_gauge *g)
{
    for (auto &kv : g->derived) cudaFree(kv.second.first);
    g->derived.clear();
}

qcd_status qcd_gauge_upload(qcd_gauge *g, const double *host, void *stream)
{
    if (!g || !host) return fail(QCD_ERR_INVALID_ARG, "gauge_upload: NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)g->lat->h * 2 * 4 * 9 * 16;
    if (!g->derived.empty()) {
        cudaStreamSynchronize(s);
        DeviceLock dl(device_mutex());
        drop_derived(g);
    }
    void *stage = nullptr;
    cudaError_t e = cudaMallocAsync(&stage, bytes, s);
    if (e != cudaSuccess) return check_cuda(e, "gauge_upload: staging");
    e = cudaMemcpyAsync(stage, host, bytes, cudaMemcpyHostToDevice, s);
    const GaugeView dst{g->data, g->lat->stride};
    if (e == cudaSuccess)
        e = launch_gauge_pack(dst, g->prec, g->recon, static_cast<const double2 *>(stage), g->lat->geom, s);
    qcd_status st = QCD_OK;
    if (e == cudaSuccess && g->recon == 8)
        st = check_recon8(dst, g->prec, static_cast<const double2 *>(stage), dst, g->prec, g->recon, g->lat->geom, s,
                          "gauge_upload");
    cudaError_t e2 = cudaFreeAsync(stage, s);
    if (e == cudaSuccess) e = e2;
    if (st != QCD_OK) return st;
    return check_cuda(e, "gauge_upload");
}

qcd_status qcd_gauge_prepare(qcd_gauge *g, qcd_prec prec, qcd_recon recon, void *stream)
{
    if (!g) return fail(QCD_ERR_INVALID_ARG, "gauge_prepare: NULL argument");
    if (!valid_prec(prec) || !valid_recon(recon)) return fail(QCD_ERR_INVALID_ARG, "gauge_prepare: bad prec/recon");
    qcd_status st;
    gauge_view(g, prec, recon, static_cast<cudaStream_t>(stream), &st);
    return st;
}

void qcd_gauge_destroy(qcd_gauge *g)
{
    if (!g) return;
    const qcd_lattice *lat = g->lat;
    {
        DeviceLock dl(device_mutex());
        cudaDeviceSynchronize();
        drop_derived(g);
        cudaFree(g->data);
        delete g;
    }
    lat_unref(lat);
}

qcd_status qcd_spinor_bytes(const qcd_lattice *lat, qcd_parity parity, qcd_prec prec, size_t *data_bytes,
                            size_t *norm_bytes)
{
    if (!lat || !data_bytes || !norm_bytes) return fail(QCD_ERR_INVALID_ARG, "spinor_bytes: NULL argument");
    if (!valid_prec(prec) || parity < 0 || parity > 2) return fail(QCD_ERR_INVALID_ARG, "spinor_bytes: bad prec/parity");
    const int nh = parity == QCD_PARITY_FULL ? 2 : 1;
    *data_bytes = nh * spinor_half_bytes(prec, lat->stride);
    *norm_bytes = nh * spinor_half_norm_bytes(prec, lat->stride);
    return QCD_OK;
}

static qcd_spinor *new_spinor(const qcd_lattice *lat, qcd_parity parity, qcd_prec prec)
{
    qcd_spinor *s = new (std::nothrow) qcd_spinor();
    if (!s) return nullptr;
    s->lat = lat;
    s->parity = parity;
    s->prec = prec;
    s->half_data_bytes = spinor_half_bytes(prec, lat->stride);
    s->half_norm_bytes = spinor_half_norm_bytes(prec, lat->stride);
    return s;
}

qcd_status qcd_spinor_create(const qcd_lattice *lat, qcd_parity parity, qcd_prec prec, qcd_spinor **out)
{
    if (!lat || !out) return fail(QCD_ERR_INVALID_ARG, "spinor_create: NULL argument");
    *out = nullptr;
    if (!valid_prec(prec) || parity < 0 || parity > 2) return fail(QCD_ERR_INVALID_ARG, "spinor_create: bad prec/parity");
    if (take_injected_failure(QCD_INJECT_SPINOR_CREATE))
        return fail(QCD_ERR_OOM, "spinor_create: injected allocation failure");
    qcd_spinor *s = new_spinor(lat, parity, prec);
    if (!s) return fail(QCD_ERR_OOM, "spinor_create: host allocation");
    const int nh = parity == QCD_PARITY_FULL ? 2 : 1;
    DeviceLock dl(device_mutex(), std::defer_lock);
    if (!lat->alloc_stream) dl.lock();
    cudaError_t e = lat_alloc(lat, &s->data, nh * s->half_data_bytes);
    if (e == cudaSuccess && s->half_norm_bytes) e = lat_alloc(lat, reinterpret_cast<void **>(&s->norm), nh * s->half_norm_bytes);
    if (e == cudaSuccess) e = lat_zero(lat, s->data, nh * s->half_data_bytes);
    if (e == cudaSuccess && s->norm) e = lat_zero(lat, s->norm, nh * s->half_norm_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        lat_free(lat, s->data);
        lat_free(lat, s->norm);
        delete s;
        return fail(QCD_ERR_OOM, "spinor_create: cudaMalloc failed");
    }
    lat_ref(lat);
    *out = s;
    return QCD_OK;
}

qcd_status qcd_spinor_create_ks(const qcd_lattice *lat, qcd_parity parity, qcd_prec prec, qcd_spinor **out)
{
    if (!lat || !out) return fail(QCD_ERR_INVALID_ARG, "spinor_create_ks: NULL argument");
    *out = nullptr;
    if (prec < QCD_PREC_F64 || prec > QCD_PREC_BF16 || parity < 0 || parity > 2)
        return fail(QCD_ERR_INVALID_ARG, "spinor_create_ks: bad prec/parity");
    qcd_spinor *s = new (std::nothrow) qcd_spinor();
    if (!s) return fail(QCD_ERR_OOM, "spinor_create_ks: host allocation");
    s->lat = lat;
    s->parity = parity;
    s->prec = prec;
    s->ks = true;
    const size_t elem = prec == QCD_PREC_F64 ? 16 : prec == QCD_PREC_F32 ? 8 : 4;
    s->half_data_bytes = 3 * elem * lat->stride;
    s->half_norm_bytes = prec == QCD_PREC_F16 ? (size_t)4 * lat->stride : 0;
    const int nh = parity == QCD_PARITY_FULL ? 2 : 1;
    DeviceLock dl(device_mutex());
    cudaError_t e = cudaMalloc(&s->data, nh * s->half_data_bytes);
    if (e == cudaSuccess && s->half_norm_bytes) e = cudaMalloc(reinterpret_cast<void **>(&s->norm), nh * s->half_norm_bytes);
    if (e == cudaSuccess) e = zero_now(s->data, nh * s->half_data_bytes);
    if (e == cudaSuccess && s->norm) e = zero_now(s->norm, nh * s->half_norm_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->data);
        cudaFree(s->norm);
        delete s;
        return fail(QCD_ERR_OOM, "spinor_create_ks: cudaMalloc failed");
    }
    lat_ref(lat);
    *out = s;
    return QCD_OK;
}

qcd_status qcd_apply_dslash_ks(const qcd_gauge *g, qcd_spinor *out, const qcd_spinor *in, void *stream)
{
    if (!g || !out || !in) return fail(QCD_ERR_INVALID_ARG, "apply_dslash_ks: NULL argument");
    if (!out->ks || !in->ks) return fail(QCD_ERR_INVALID_ARG, "apply_dslash_ks: fields must be staggered");
    if (out->lat != g->lat || in->lat != g->lat) return fail(QCD_ERR_INVALID_ARG, "apply_dslash_ks: lattices differ");
    if (out->prec != in->prec) return fail(QCD_ERR_INVALID_ARG, "apply_dslash_ks: precisions differ");
    if (out->data == in->data) return fail(QCD_ERR_INVALID_ARG, "apply_dslash_ks: out aliases in");
    const bool both = out->parity == QCD_PARITY_FULL && in->parity == QCD_PARITY_FULL;
    if (!both && !(out->parity != QCD_PARITY_FULL && in->parity == 1 - out->parity))
        return fail(QCD_ERR_INVALID_ARG, "apply_dslash_ks: parities must be (EVEN, ODD), (ODD, EVEN) or (FULL, FULL)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    qcd_status st;
    GaugeView U = gauge_view(g, out->prec, g->recon, s, &st);
    if (st != QCD_OK) return st;
    const FieldView fo = view_of(out), fi = view_of(in);
    KsLaunch a;
    memset(&a, 0, sizeof(a));
    a.g = g->lat->geom;
    a.both = both ? 1 : 0;
    a.out_parity = both ? 0 : out->parity;
    a.U = U;
    if (both) {
        for (int p = 0; p < 2; ++p) {
            a.out[p] = fo.hv[p];
            a.in[p] = fi.hv[1 - p];
        }
    } else {
        a.out[a.out_parity] = fo.hv[0];
        a.in[a.out_parity] = fi.hv[0];
    }
    return check_cuda(launch_dslash_ks(out->prec, g->recon, a, s), "apply_dslash_ks");
}

qcd_status qcd_spinor_wrap_device(const qcd_lattice *lat, qcd_parity parity, qcd_prec prec, void *data, void *norm,
                                  qcd_spinor **out)
{
    if (!lat || !out || !data) return fail(QCD_ERR_INVALID_ARG, "spinor_wrap_device: NULL argument");
    *out = nullptr;
    if (!valid_prec(prec) || parity < 0 || parity > 2) return fail(QCD_ERR_INVALID_ARG, "spinor_wrap_device: bad prec/parity");
    if (prec == QCD_PREC_F16 && !norm) return fail(QCD_ERR_INVALID_ARG, "spinor_wrap_device: F16 needs a norm buffer");
    if ((reinterpret_cast<uintptr_t>(data) & 255) || (reinterpret_cast<uintptr_t>(norm) & 255))
        return fail(QCD_ERR_INVALID_ARG, "spinor_wrap_device: buffers must be 256-byte aligned");
    qcd_spinor *s = new_spinor(lat, parity, prec);
    if (!s) return fail(QCD_ERR_OOM, "spinor_wrap_device: host allocation");
    s->data = data;
    s->norm = prec == QCD_PREC_F16 ? static_cast<float *>(norm) : nullptr;
    s->owns = false;
    lat_ref(lat);
    *out = s;
    return QCD_OK;
}

void qcd_spinor_destroy(qcd_spinor *s)
{
    if (!s) return;
    const qcd_lattice *lat = s->lat;
    if (s->owns && lat->alloc_stream) {
        // stream-ordered lattice: freed after the work queued on its stream
        lat_free(lat, s->data);
        lat_free(lat, s->norm);
    } else if (s->owns) {
        DeviceLock dl(device_mutex());
        cudaDeviceSynchronize();
        cudaFree(s->data);
        cudaFree(s->norm);
    }
    delete s;
    lat_unref(lat);
}

qcd_status qcd_spinor_upload(qcd_spinor *s, const double *host, void *stream)
{
    if (!s || !host) return fail(QCD_ERR_INVALID_ARG, "spinor_upload: NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nh = s->parity == QCD_PARITY_FULL ? 2 : 1;
    const size_t bytes = (size_t)nh * s->lat->h * (s->ks ? 48 : 192);
    if (s->ks) {
        void *stage = workspace(s->lat, "staging", bytes);
        if (!stage) return fail(QCD_ERR_OOM, "spinor_upload: staging");
        cudaError_t e = cudaMemcpyAsync(stage, host, bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_ks_pack(view_of(s), s->parity, static_cast<const double2 *>(stage), s->lat->geom, st);
        return check_cuda(e, "spinor_upload");
    }
    void *stage = workspace(s->lat, "staging", bytes);
    if (!stage) return fail(QCD_ERR_OOM, "spinor_upload: staging");
    cudaError_t e = cudaMemcpyAsync(stage, host, bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_spinor_pack(view_of(s), s->parity, static_cast<const double2 *>(stage), s->lat->geom, st);
    return check_cuda(e, "spinor_upload");
}

qcd_status qcd_spinor_download(const qcd_spinor *s, double *host, void *stream)
{
    if (!s || !host) return fail(QCD_ERR_INVALID_ARG, "spinor_download: NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nh = s->parity == QCD_PARITY_FULL ? 2 : 1;
    const size_t bytes = (size_t)nh * s->lat->h * (s->ks ? 48 : 192);
    if (s->ks) {
        void *stage = workspace(s->lat, "staging", bytes);
        if (!stage) return fail(QCD_ERR_OOM, "spinor_download: staging");
        cudaError_t e = launch_ks_unpack(static_cast<double2 *>(stage), view_of(s), s->parity, s->lat->geom, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host, stage, bytes, cudaMemcpyDeviceToHost, st);
        return check_cuda(e, "spinor_download");
    }
    void *stage = workspace(s->lat, "staging", bytes);
    if (!stage) return fail(QCD_ERR_OOM, "spinor_download: staging");
    cudaError_t e = launch_spinor_unpack(static_cast<double2 *>(stage), view_of(s), s->parity, s->lat->geom, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, stage, bytes, cudaMemcpyDeviceToHost, st);
    return check_cuda(e, "spinor_download");
}

qcd_status qcd_spinor_zero(qcd_spinor *s, void *stream)
{
    if (!s) return fail(QCD_ERR_INVALID_ARG, "spinor_zero: NULL argument");
    if (s->ks) return fail(QCD_ERR_INVALID_ARG, "spinor_zero: not defined for staggered fields");
    return check_cuda(launch_zero(view_of(s), static_cast<cudaStream_t>(stream)), "spinor_zero");
}

qcd_status qcd_spinor_convert(qcd_spinor *dst, const qcd_spinor *src, void *stream)
{
    if (!dst || !src) return fail(QCD_ERR_INVALID_ARG, "spinor_convert: NULL argument");
    if (dst->lat != src->lat || dst->parity != src->parity)
        return fail(QCD_ERR_INVALID_ARG, "spinor_convert: lattice or parity differ");
    if (dst->ks || src->ks) return fail(QCD_ERR_INVALID_ARG, "spinor_convert: not defined for staggered fields");
    return check_cuda(launch_convert(view_of(dst), view_of(src), static_cast<cudaStream_t>(stream)), "spinor_convert");
}

qcd_status qcd_spinor_norm2(const qcd_spinor *s, double *result_device, void *stream)
{
    if (!s || !result_device) return fail(QCD_ERR_INVALID_ARG, "spinor_norm2: NULL argument");
    if (s->ks) return fail(QCD_ERR_INVALID_ARG, "spinor_norm2: not defined for staggered fields");
    return check_cuda(launch_norm2(view_of(s), reduction_of(s->lat), FIN_STORE, s->lat->state, result_device,
                                   static_cast<cudaStream_t>(stream)),
                      "spinor_norm2");
}

qcd_status qcd_apply_dslash(const qcd_gauge *g, qcd_spinor *out, const qcd_spinor *in, int dagger, void *stream)
{
    if (!g || !out || !in) return fail(QCD_ERR_INVALID_ARG, "apply_dslash: NULL argument");
    if (out->lat != g->lat || in->lat != g->lat) return fail(QCD_ERR_INVALID_ARG, "apply_dslash: lattices differ");
    if (out->prec != in->prec) return fail(QCD_ERR_INVALID_ARG, "apply_dslash: precisions differ");
    if (out->ks || in->ks) return fail(QCD_ERR_INVALID_ARG, "apply_dslash: staggered fields need qcd_apply_dslash_ks");
    if (out == in || out->data == in->data) return fail(QCD_ERR_INVALID_ARG, "apply_dslash: out aliases in");
    const bool both = out->parity == QCD_PARITY_FULL && in->parity == QCD_PARITY_FULL;
    if (!both && !(out->parity != QCD_PARITY_FULL && in->parity == 1 - out->parity))
        return fail(QCD_ERR_INVALID_ARG, "apply_dslash: parities must be (EVEN, ODD), (ODD, EVEN) or (FULL, FULL)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    qcd_status st;
    GaugeView U = gauge_view(g, out->prec, g->recon, s, &st);
    if (st != QCD_OK) return st;
    const FieldView fo = view_of(out), fi = view_of(in);
    HopArgs h{};
    h.out = &fo;
    h.in = &fi;
    h.y = nullptr;
    h.out_parity = both ? 0 : out->parity;
    h.both = both;
    h.dagger = dagger ? 1 : 0;
    h.plain = true;
    h.fin = FIN_STORE;
    return check_cuda(hop(g->lat, U, g->recon, h, s), "apply_dslash");
}

qcd_status qcd_apply_dslash_multi(const qcd_gauge *g, qcd_spinor *const *out, const qcd_spinor *const *in, int nrhs,
                                  int dagger, void *stream)
{
    if (!g || !out || !in) return fail(QCD_ERR_INVALID_ARG, "apply_dslash_multi: NULL argument");
    if (nrhs < 1 || nrhs > kMaxRhs) return fail(QCD_ERR_INVALID_ARG, "apply_dslash_multi: nrhs = %d not in 1..%d", nrhs, kMaxRhs);
    for (int k = 0; k < nrhs; ++k) {
        if (!out[k] || !in[k]) return fail(QCD_ERR_INVALID_ARG, "apply_dslash_multi: NULL field");
        if (out[k]->lat != g->lat || in[k]->lat != g->lat) return fail(QCD_ERR_INVALID_ARG, "apply_dslash_multi: lattices differ");
        if (out[k]->prec != in[0]->prec || in[k]->prec != in[0]->prec || out[k]->parity != out[0]->parity ||
            in[k]->parity != in[0]->parity)
            return fail(QCD_ERR_INVALID_ARG, "apply_dslash_multi: fields must share precision and parity");
        if (out[k]->data == in[k]->data) return fail(QCD_ERR_INVALID_ARG, "apply_dslash_multi: out aliases in");
    }
    const bool both = out[0]->parity == QCD_PARITY_FULL && in[0]->parity == QCD_PARITY_FULL;
    if (!both && !(out[0]->parity != QCD_PARITY_FULL && in[0]->parity == 1 - out[0]->parity))
        return fail(QCD_ERR_INVALID_ARG, "apply_dslash_multi: parities must be (EVEN, ODD), (ODD, EVEN) or (FULL, FULL)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const qcd_lattice *lat = g->lat;
    qcd_status st;
    GaugeView U = gauge_view(g, in[0]->prec, g->recon, s, &st);
    if (st != QCD_OK) return st;
    int L = 0;
    while ((1 << L) < nrhs) ++L;
    const int nh = both ? 2 : 1, prec = in[0]->prec;
    const FieldView bi = ws_field(lat, "dm_in", nh, prec, L), bo = ws_field(lat, "dm_out", nh, prec, L);
    if (!bi.hv[0].data || !bo.hv[0].data) return fail(QCD_ERR_OOM, "apply_dslash_multi: workspace");
    cudaError_t e = launch_zero(bi, s);
    FieldView pv[kMaxRhs];
    for (int k = 0; k < nrhs; ++k) pv[k] = view_of(in[k]);
    if (e == cudaSuccess) e = launch_batch_copy(bi, pv, nrhs, 1, s);
    if (e != cudaSuccess) return check_cuda(e, "apply_dslash_multi: gather");
    HopArgs h{};
    h.out = &bo;
    h.in = &bi;
    h.out_parity = both ? 0 : out[0]->parity;
    h.both = both;
    h.dagger = dagger ? 1 : 0;
    h.plain = true;
    h.fin = FIN_STORE;
    e = hop(lat, U, g->recon, h, s);
    for (int k = 0; k < nrhs; ++k) pv[k] = view_of(out[k]);
    if (e == cudaSuccess) e = launch_batch_copy(bo, pv, nrhs, 0, s);
    return check_cuda(e, "apply_dslash_multi");
}

qcd_status qcd_apply_M(const qcd_gauge *g, qcd_spinor *out, const qcd_spinor *in, double kappa, double mu, int eo,
                       int dagger, void *stream)
{
    if (!g || !out || !in) return fail(QCD_ERR_INVALID_ARG, "apply_M: NULL argument");
    if (out->lat != g->lat || in->lat != g->lat) return fail(QCD_ERR_INVALID_ARG, "apply_M: lattices differ");
    if (out->prec != in->prec) return fail(QCD_ERR_INVALID_ARG, "apply_M: precisions differ");
    if (out->ks || in->ks) return fail(QCD_ERR_INVALID_ARG, "apply_M: not defined for staggered fields");
    if (out == in || out->data == in->data) return fail(QCD_ERR_INVALID_ARG, "apply_M: out aliases in");
    if (eo && (out->parity != QCD_PARITY_EVEN || in->parity != QCD_PARITY_EVEN))
        return fail(QCD_ERR_INVALID_ARG, "apply_M: eo = 1 needs EVEN fields");
    if (!eo && (out->parity != QCD_PARITY_FULL || in->parity != QCD_PARITY_FULL))
        return fail(QCD_ERR_INVALID_ARG, "apply_M: eo = 0 needs FULL fields");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    qcd_status st;
    GaugeView U = gauge_view(g, out->prec, g->recon, s, &st);
    if (st != QCD_OK) return st;
    const double a = 2.0 * kappa * mu, b = dagger ? -a : a;
    const bool tw = a != 0.0;
    const FieldView fo = view_of(out), fi = view_of(in);
    HopArgs h{};
    h.dagger = dagger ? 1 : 0;
    h.fin = FIN_STORE;
    if (!eo) {
        h.out = &fo;
        h.in = &fi;
        h.y = &fi;
        h.both = true;
        h.cy = coef_twist(b);
        h.cd = coef_real(-kappa);
        h.twisted = tw;
        return check_cuda(hop(g->lat, U, g->recon, h, s), "apply_M");
    }
    const FieldView t = ws_field(g->lat, "applyM_t", 1, out->prec);
    if (!t.hv[0].data) return fail(QCD_ERR_OOM, "apply_M: workspace");
    h.out = &t;
    h.in = &fi;
    h.y = nullptr;
    h.out_parity = 1;
    h.plain = !tw;
    h.twisted = tw;
    h.cd = coef_twist_inv(b);
    cudaError_t e = hop(g->lat, U, g->recon, h, s);
    if (e != cudaSuccess) return check_cuda(e, "apply_M");
    HopArgs h2{};
    h2.dagger = h.dagger;
    h2.fin = FIN_STORE;
    h2.out = &fo;
    h2.in = &t;
    h2.y = &fi;
    h2.out_parity = 0;
    h2.cy = coef_twist(b);
    h2.cd = coef_real(-kappa * kappa);
    h2.twisted = tw;
    return check_cuda(hop(g->lat, U, g->recon, h2, s), "apply_M");
}

}  // extern "C"
