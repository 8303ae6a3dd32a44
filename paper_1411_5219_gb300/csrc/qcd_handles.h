// Handle structures behind the opaque C types (internal).
#pragma once

#include <atomic>
#include <map>
#include <mutex>
#include <shared_mutex>
#include <string>

#include "qcd_ops.h"

// Doubles of the pinned coefficient staging buffer: 96 per rhs, up to 32 rhs.
constexpr int kCoefHostDoubles = 96 * 32 * 3 / 2;

struct qcd_lattice {
    int dims[4];
    int t_bc;
    int device;
    qcd::Geom geom;
    int h;       // sites per parity
    int stride;  // padded sites per plane

    // Scratch shared by the calls on this lattice (stream-ordered use).
    double *red_partials = nullptr;  // reduction partials
    size_t red_cap = 0;              // doubles
    unsigned *red_counter = nullptr; // ticket counter (zero between kernels)
    double *red_out = nullptr;       // FIN_STORE results (8 doubles)
    double *red_out_big = nullptr;   // per-rhs FIN_STORE results (2 * kMaxRhs doubles)
    qcd::CgState *state = nullptr;   // device CG state
    qcd::CgState *state_host = nullptr;  // pinned mirror
    double *coef_host = nullptr;         // pinned staging of a solve's coefficient table (kCoefHostDoubles)
    // Named workspace buffers (staging, solver fields), grown on demand.
    mutable std::map<std::string, std::pair<void *, size_t>> ws;
    // Instantiated CG-loop graphs keyed by solver configuration and field
    // addresses, and the stream used only to capture them.
    struct GraphEntry {
        cudaGraph_t graph;
        cudaGraphExec_t exec;
        unsigned long long last_use;
    };
    mutable std::map<std::string, GraphEntry> graphs;
    mutable unsigned long long graph_clock = 0;
    mutable cudaStream_t capture_stream = nullptr;
    // Stream-ordered memory (set for the solve server's contexts): device
    // buffers of this lattice, its workspace and its spinors are allocated
    // with cudaMallocAsync and freed with cudaFreeAsync on this stream, and
    // the pinned staging comes from a reuse pool, so creating, growing and
    // destroying them never synchronises the whole device.  Every use must
    // then be ordered after `alloc_stream` (the server uses this stream only).
    cudaStream_t alloc_stream = nullptr;
    // Held by the creator and by every gauge field and spinor on the
    // lattice: qcd_lattice_destroy drops the creator's reference and the
    // lattice is freed with the last one, so fields may be destroyed after
    // their lattice in any order.
    mutable std::atomic<int> refs{1};
};

struct qcd_gauge {
    const qcd_lattice *lat;
    int prec, recon;
    void *data = nullptr;
    size_t bytes = 0;
    // Copies in other (prec, recon) formats, keyed by prec * 100 + recon.
    std::map<int, std::pair<void *, size_t>> derived;
};

struct qcd_spinor {
    const qcd_lattice *lat;
    int parity;  // qcd_parity
    int prec;
    void *data = nullptr;
    float *norm = nullptr;
    size_t half_data_bytes = 0;  // bytes of one half field's planes
    size_t half_norm_bytes = 0;
    bool owns = true;
    bool ks = false;  // staggered field: 3 complex per site
};

namespace qcd {

// Graph capture vs device-wide operations.  A CUDA graph capture on one
// thread is invalidated when another thread synchronises the whole device or
// frees memory meanwhile.  Captures hold this lock shared (several may run
// at once); every call that allocates, frees or synchronises the device
// holds it exclusively.
std::shared_mutex &device_mutex();
using CaptureLock = std::shared_lock<std::shared_mutex>;
using DeviceLock = std::unique_lock<std::shared_mutex>;

// True inside a qcd_profile_begin/end window (per-launch events cannot be
// captured into conditional graph bodies, so the solver runs eagerly then).
bool profiling_active();

// Per-thread error message for qcd_last_error().
qcd_status fail(qcd_status code, const char *fmt, ...);
qcd_status check_cuda(cudaError_t e, const char *what);

size_t spinor_half_bytes(int prec, int stride);
size_t spinor_half_norm_bytes(int prec, int stride);
size_t gauge_bytes(int prec, int recon, int stride);

// Workspace buffer `name` of at least `bytes` on the lattice.
void *workspace(const qcd_lattice *lat, const std::string &name, size_t bytes);

// A lattice (and, through qcd_spinor_create on it, its spinors) whose device
// memory is stream-ordered on `s` (see qcd_lattice::alloc_stream).
qcd_status lattice_create_on(const int dims[4], int t_bc, cudaStream_t s, qcd_lattice **out);

// Views.
FieldView view_of(const qcd_spinor *s);
FieldView view_half(const qcd_spinor *s, int half);  // half of a FULL field
FieldView ws_field(const qcd_lattice *lat, const std::string &name, int nh, int prec, int rhs_log2 = 0);
GaugeView gauge_view(const qcd_gauge *g, int prec, int recon, cudaStream_t s, qcd_status *st);
Reduction reduction_of(const qcd_lattice *lat);

cudaError_t launch_dslash(int prec, int recon, const DslashLaunch &a, cudaStream_t s);

// Chiral coefficients of (1 + i b gamma_5) and of its inverse.
struct Coef {
    double c[2][2];  // [chirality][re, im]
};
Coef coef_twist(double b);
Coef coef_twist_inv(double b);
Coef coef_scale(Coef c, double s);
Coef coef_real(double s);

// Dslash launch on FieldViews: out (parity p) = cy .* y + cd .* D in.
// `y` may be null.  With both = true, out, in and y are FULL fields.
struct HopArgs {
    const FieldView *out, *in, *y;
    int out_parity;
    bool both;
    int dagger;
    Coef cy, cd;
    bool plain;      // out = D in (cy, cd ignored)
    bool twisted;    // complex chiral coefficients
    bool reduce;
    FinalizeKind fin;
    bool check_status;
    const Reduction *red;  // scratch of the fused reduction (nullptr: the lattice's)
    const double *coef;    // device table of cy, cd (8 doubles) read at run time, or nullptr
    const float *coef_f;   // its float image (same layout; required with coef)
    int coef_stride;       // doubles between the tables of consecutive rhs (0: shared)
    int run_status;        // with check_status: run only under this CG status (default CG_RUNNING = 0)
};
cudaError_t hop(const qcd_lattice *lat, const GaugeView &U, int recon, const HopArgs &h, cudaStream_t s);

// The CG solve behind qcd_solve_cg / qcd_solve_cg_multi, with an optional
// context lattice (scratch, state, graphs) other than the gauge field's.
// prm holds one parameter set per right-hand side (kappa, mu and tol may
// differ; the other fields must agree).
qcd_status solve_impl(const qcd_gauge *g, qcd_spinor *const *x, const qcd_spinor *const *b, int nrhs,
                      const qcd_solver_params *prm, qcd_solver_stats *stats, cudaStream_t s, const qcd_lattice *ctx);

// Autotuned threads per block of the hopping kernel for this configuration
// (times the candidates on first use outside stream capture).
int tuned_tpb(const qcd_lattice *lat, const GaugeView &U, int prec, int recon, int rhs_log2, bool both, cudaStream_t s);

}  // namespace qcd
