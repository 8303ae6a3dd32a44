// Solve server: a request loop that admits CG solves as slots and device
// memory free up and runs them concurrently on the GPU.
//
// The paper points out that finite-temperature studies form a naturally
// parallel setup of many independent simulations over couplings and volumes
// (Sec. 1), and that device memory bounds what can run (Sec. 2).  Here many
// independent inversions of different volumes and hopping parameters share
// one GPU:
//   * gauge fields stay resident (registered once, shared read-only);
//   * `slots` worker threads each own a CUDA stream and, per lattice volume,
//     a solver context (lattice scratch, CG state, cached CG graph, device
//     b and x);
//   * requests queue in arrival order; the head request is admitted to a
//     free slot as soon as the memory its context needs fits the budget
//     (idle contexts of that slot are released to make room), so requests
//     that arrive while others run start as soon as a slot and memory free
//     up, and their kernels overlap with the running ones on the device;
//   * each request records submit, start and end times for latency.
// Results do not depend on what else runs: a solve's kernels, launch shapes
// and fixed-order reductions are the same alone and in the mix.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "qcd_handles.h"

namespace {

using clock_type = std::chrono::steady_clock;

struct VolumeCtx {
    qcd_lattice *lat = nullptr;
    qcd_spinor *b = nullptr, *x = nullptr;
    std::vector<std::pair<qcd_spinor *, qcd_spinor *>> more;  // b, x of further systems of a batch
    size_t reserved = 0;  // bytes counted against the budget
};

struct Job {
    long long id;
    qcd_request req;
    double t_submit = 0, t_start = 0, t_end = 0;
    int status = QCD_OK;
    int slot = -1;
    qcd_solver_stats stats{};
    bool done = false;
};

std::string dims_key(const qcd_lattice *l)
{
    return std::to_string(l->dims[0]) + "x" + std::to_string(l->dims[1]) + "x" + std::to_string(l->dims[2]) + "x" +
           std::to_string(l->dims[3]) + (l->t_bc < 0 ? "a" : "p");
}

// Device bytes of one solver context: b, x (FULL FP64) and the solver's
// workspace (FP64 and inner fields, operator temporaries, residual fields,
// staging), bounded by 24 FP64 full fields.
size_t context_bytes(const qcd_lattice *l) { return (size_t)24 * 2 * l->h * 192; }

// Volumes up to 24^3 x 8 sites count as small (high-priority stream).
constexpr size_t kSmallVolume = 24 * 24 * 24 * 8;

}  // namespace

struct qcd_server {
    int device = 0;
    size_t budget = 0, used = 0;
    int nslots = 0;
    int batch_small = 0;  // sites at most, for batching small requests (0: off)
    clock_type::time_point t0;
    std::vector<const qcd_gauge *> gauges;
    std::deque<Job *> queue;
    std::map<long long, Job *> jobs;
    long long next_id = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_idle;
    bool stop = false;
    int waiters = 0;  // threads inside qcd_server_wait
    std::vector<std::thread> workers;
    std::vector<std::map<std::string, VolumeCtx>> slot_ctx;
    std::vector<cudaStream_t> streams;     // per slot, high priority (small volumes)
    std::vector<cudaStream_t> streams_lo;  // per slot, low priority (large volumes)
    std::vector<int> busy;

    double now() const { return std::chrono::duration<double>(clock_type::now() - t0).count(); }
};

namespace {

void release(qcd_server *sv, VolumeCtx &c)
{
    for (auto &bx : c.more) {
        qcd_spinor_destroy(bx.first);
        qcd_spinor_destroy(bx.second);
    }
    qcd_spinor_destroy(c.b);
    qcd_spinor_destroy(c.x);
    qcd_lattice_destroy(c.lat);
    sv->used -= c.reserved;
    c = VolumeCtx{};
}

// Under sv->mu: can slot `s` take job `j` now?  Reserves memory if so.
bool admit(qcd_server *sv, int s, Job *j)
{
    const qcd_lattice *gl = sv->gauges[j->req.gauge_id]->lat;
    const std::string key = dims_key(gl);
    auto &ctxs = sv->slot_ctx[s];
    if (ctxs.count(key)) return true;
    const size_t need = context_bytes(gl);
    // release this slot's idle contexts of other volumes until it fits
    for (auto it = ctxs.begin(); sv->used + need > sv->budget && it != ctxs.end();) {
        release(sv, it->second);
        it = ctxs.erase(it);
    }
    if (sv->used + need > sv->budget) return false;
    sv->used += need;
    ctxs[key].reserved = need;
    return true;
}

void run_job(qcd_server *sv, int s, Job *j)
{
    cudaSetDevice(sv->device);
    const qcd_gauge *g = sv->gauges[j->req.gauge_id];
    VolumeCtx *c;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        c = &sv->slot_ctx[s][dims_key(g->lat)];
    }
    qcd_status st = QCD_OK;
    // Small volumes run on the slot's high-priority stream, so their few
    // short kernels are not queued behind the long ones of large volumes.
    // The context's device memory is stream-ordered on that stream: building
    // or releasing a context never synchronises the other slots' work.
    cudaStream_t stream = (size_t)g->lat->h * 2 <= kSmallVolume ? sv->streams[s] : sv->streams_lo[s];
    if (!c->lat || !c->b || !c->x) {
        // build the context whole; a part left by an earlier failed build is
        // dropped first, and a failed build leaves nothing behind (the
        // reserved bytes stay with the context entry until it is released)
        qcd_spinor_destroy(c->b);
        qcd_spinor_destroy(c->x);
        qcd_lattice_destroy(c->lat);
        c->lat = nullptr;
        c->b = c->x = nullptr;
        st = qcd::lattice_create_on(g->lat->dims, g->lat->t_bc, stream, &c->lat);
        if (st == QCD_OK) st = qcd_spinor_create(c->lat, QCD_PARITY_FULL, QCD_PREC_F64, &c->b);
        if (st == QCD_OK) st = qcd_spinor_create(c->lat, QCD_PARITY_FULL, QCD_PREC_F64, &c->x);
        if (st != QCD_OK) {
            qcd_spinor_destroy(c->b);
            qcd_spinor_destroy(c->x);
            qcd_lattice_destroy(c->lat);
            c->lat = nullptr;
            c->b = c->x = nullptr;
        }
    }
    if (st == QCD_OK) st = qcd_spinor_upload(c->b, j->req.b_host, stream);
    if (st == QCD_OK) {
        const qcd_request &r = j->req;
        qcd_solver_params prm{r.kappa, r.mu, r.tol, r.maxiter, 1, 0, r.inner_prec, r.inner_recon, r.reliable_delta};
        qcd_spinor *xs[1] = {c->x};
        const qcd_spinor *bs[1] = {c->b};
        st = qcd::solve_impl(g, xs, bs, 1, &prm, &j->stats, stream, c->lat);
        // NOT_CONVERGED still returns x
        if (st == QCD_OK || st == QCD_ERR_NOT_CONVERGED) {
            qcd_status st2 = qcd_spinor_download(c->x, j->req.x_host, stream);
            if (st2 == QCD_OK) st2 = qcd_stream_sync(stream);
            if (st2 != QCD_OK) st = st2;
        }
    }
    j->status = st;
}

// Small requests taken together: one persistent launch solves them all
// (qcd_solve_cg_many); each keeps its own b and x on its volume's context.
void run_batch(qcd_server *sv, int s, std::vector<Job *> &jobs)
{
    cudaSetDevice(sv->device);
    const int n = (int)jobs.size();
    cudaStream_t stream = sv->streams[s];
    std::vector<const qcd_gauge *> g(n);
    std::vector<qcd_spinor *> xs(n);
    std::vector<const qcd_spinor *> bs(n);
    std::vector<qcd_solver_params> prm(n);
    std::map<std::string, int> used;  // systems per volume so far
    qcd_status st = QCD_OK;
    for (int k = 0; k < n && st == QCD_OK; ++k) {
        Job *j = jobs[k];
        g[k] = sv->gauges[j->req.gauge_id];
        VolumeCtx *c;
        const std::string key = dims_key(g[k]->lat);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            c = &sv->slot_ctx[s][key];
        }
        if (!c->lat || !c->b || !c->x) {
            for (auto &bx : c->more) {
                qcd_spinor_destroy(bx.first);
                qcd_spinor_destroy(bx.second);
            }
            c->more.clear();
            qcd_spinor_destroy(c->b);
            qcd_spinor_destroy(c->x);
            qcd_lattice_destroy(c->lat);
            c->lat = nullptr;
            c->b = c->x = nullptr;
            st = qcd::lattice_create_on(g[k]->lat->dims, g[k]->lat->t_bc, stream, &c->lat);
            if (st == QCD_OK) st = qcd_spinor_create(c->lat, QCD_PARITY_FULL, QCD_PREC_F64, &c->b);
            if (st == QCD_OK) st = qcd_spinor_create(c->lat, QCD_PARITY_FULL, QCD_PREC_F64, &c->x);
            if (st != QCD_OK) break;
        }
        const int o = used[key]++;
        if (o == 0) {
            bs[k] = c->b;
            xs[k] = c->x;
        } else {
            while ((int)c->more.size() < o) {
                qcd_spinor *b2 = nullptr, *x2 = nullptr;
                st = qcd_spinor_create(c->lat, QCD_PARITY_FULL, QCD_PREC_F64, &b2);
                if (st == QCD_OK) st = qcd_spinor_create(c->lat, QCD_PARITY_FULL, QCD_PREC_F64, &x2);
                if (st != QCD_OK) {
                    qcd_spinor_destroy(b2);
                    qcd_spinor_destroy(x2);
                    break;
                }
                c->more.emplace_back(b2, x2);
            }
            if (st != QCD_OK) break;
            bs[k] = c->more[o - 1].first;
            xs[k] = c->more[o - 1].second;
        }
        st = qcd_spinor_upload(const_cast<qcd_spinor *>(bs[k]), j->req.b_host, stream);
        const qcd_request &r = j->req;
        prm[k] = qcd_solver_params{r.kappa, r.mu, r.tol, r.maxiter, 1, 0, (qcd_prec)QCD_PREC_F64, (qcd_recon)18, r.reliable_delta};
    }
    std::vector<qcd_solver_stats> stats(n);
    // the full resident grid (capped at 32 blocks, to start sooner beside
    // the other slots' kernels, it served 8^3x4 requests at half the rate)
    if (st == QCD_OK)
        st = qcd_solve_cg_many(n, g.data(), xs.data(), bs.data(), prm.data(), stats.data(), 0, 0, stream);
    const bool ran = st == QCD_OK || st == QCD_ERR_NOT_CONVERGED || st == QCD_ERR_BREAKDOWN;
    qcd_status st2 = QCD_OK;
    if (ran)
        for (int k = 0; k < n && st2 == QCD_OK; ++k) st2 = qcd_spinor_download(xs[k], jobs[k]->req.x_host, stream);
    if (st2 == QCD_OK) st2 = qcd_stream_sync(stream);
    for (int k = 0; k < n; ++k) {
        Job *j = jobs[k];
        j->stats = stats[k];
        if (!ran || st2 != QCD_OK)
            j->status = st2 != QCD_OK ? st2 : st;
        else  // per system: converged to its own target, else the batch's error
            j->status = st == QCD_OK || stats[k].true_rel_residual <= j->req.tol ? QCD_OK : st;
    }
}

bool small_job(const qcd_server *sv, const Job *j)
{
    return sv->batch_small > 0 && (long long)sv->gauges[j->req.gauge_id]->lat->h * 2 <= sv->batch_small;
}

void worker(qcd_server *sv, int s)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        sv->cv_work.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
        if (sv->stop) return;
        Job *j = sv->queue.front();
        if (!admit(sv, s, j)) {  // wait for memory to free up, then retry
            sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            continue;
        }
        sv->queue.pop_front();
        sv->busy[s] = 1;
        std::vector<Job *> batch{j};
        if (small_job(sv, j)) {
            // further small requests queued behind it, in order, while their
            // contexts fit (same maxiter: one launch iterates them together)
            for (auto it = sv->queue.begin(); it != sv->queue.end() && batch.size() < 16;) {
                Job *c = *it;
                if (!small_job(sv, c) || c->req.maxiter != j->req.maxiter) {
                    ++it;
                    continue;
                }
                if (!admit(sv, s, c)) break;
                batch.push_back(c);
                it = sv->queue.erase(it);
            }
        }
        const double t = sv->now();
        for (Job *b : batch) {
            b->slot = s;
            b->t_start = t;
        }
        lk.unlock();
        if (batch.size() == 1 && !small_job(sv, j))
            run_job(sv, s, j);
        else
            run_batch(sv, s, batch);
        lk.lock();
        const double te = sv->now();
        for (Job *b : batch) {
            b->t_end = te;
            b->done = true;
        }
        sv->busy[s] = 0;
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

}  // namespace

using qcd::fail;

extern "C" {

qcd_status qcd_server_create(const qcd_server_config *cfg, qcd_server **out)
{
    if (!cfg || !out) return fail(QCD_ERR_INVALID_ARG, "server_create: NULL argument");
    *out = nullptr;
    if (cfg->slots < 1 || cfg->slots > 64 || cfg->memory_budget == 0)
        return fail(QCD_ERR_INVALID_ARG, "server_create: slots must be 1..64 and the budget positive");
    auto *sv = new (std::nothrow) qcd_server();
    if (!sv) return fail(QCD_ERR_OOM, "server_create: host allocation");
    cudaGetDevice(&sv->device);
    sv->budget = cfg->memory_budget;
    sv->nslots = cfg->slots;
    sv->batch_small = cfg->batch_small_sites > 0 ? cfg->batch_small_sites : 0;
    sv->t0 = clock_type::now();
    sv->slot_ctx.resize(cfg->slots);
    sv->busy.assign(cfg->slots, 0);
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    for (int s = 0; s < cfg->slots; ++s) {
        cudaStream_t hi = nullptr, lo = nullptr;
        if (cudaStreamCreateWithPriority(&hi, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&lo, cudaStreamNonBlocking, prio_lo) != cudaSuccess) {
            if (hi) cudaStreamDestroy(hi);
            for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
            for (cudaStream_t x : sv->streams_lo) cudaStreamDestroy(x);
            delete sv;
            return fail(QCD_ERR_CUDA, "server_create: cudaStreamCreate failed");
        }
        sv->streams.push_back(hi);
        sv->streams_lo.push_back(lo);
    }
    for (int s = 0; s < cfg->slots; ++s) sv->workers.emplace_back(worker, sv, s);
    *out = sv;
    return QCD_OK;
}

qcd_status qcd_server_add_gauge(qcd_server *sv, const qcd_gauge *g, int *gauge_id)
{
    if (!sv || !g || !gauge_id) return fail(QCD_ERR_INVALID_ARG, "server_add_gauge: NULL argument");
    if (g->prec != QCD_PREC_F64) return fail(QCD_ERR_INVALID_ARG, "server_add_gauge: the gauge field must be F64");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->gauges.push_back(g);
    *gauge_id = (int)sv->gauges.size() - 1;
    return QCD_OK;
}

qcd_status qcd_server_submit(qcd_server *sv, const qcd_request *req, long long *request_id)
{
    if (!sv || !req || !request_id) return fail(QCD_ERR_INVALID_ARG, "server_submit: NULL argument");
    if (!req->b_host || !req->x_host) return fail(QCD_ERR_INVALID_ARG, "server_submit: NULL host buffer");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return fail(QCD_ERR_INVALID_ARG, "server_submit: the server is being destroyed");
    if (req->gauge_id < 0 || req->gauge_id >= (int)sv->gauges.size())
        return fail(QCD_ERR_INVALID_ARG, "server_submit: unknown gauge id %d", req->gauge_id);
    if (context_bytes(sv->gauges[req->gauge_id]->lat) > sv->budget)
        return fail(QCD_ERR_OOM, "server_submit: the request needs more device memory than the whole budget");
    Job *j = new Job();
    j->id = sv->next_id++;
    j->req = *req;
    j->t_submit = sv->now();
    sv->jobs[j->id] = j;
    sv->queue.push_back(j);
    *request_id = j->id;
    sv->cv_work.notify_all();
    return QCD_OK;
}

qcd_status qcd_server_wait(qcd_server *sv, long long request_id, qcd_request_result *out)
{
    if (!sv || !out) return fail(QCD_ERR_INVALID_ARG, "server_wait: NULL argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(request_id);
    if (it == sv->jobs.end()) return fail(QCD_ERR_INVALID_ARG, "server_wait: unknown request %lld", request_id);
    Job *j = it->second;
    ++sv->waiters;
    sv->cv_done.wait(lk, [&] { return j->done; });
    --sv->waiters;
    out->id = j->id;
    out->status = j->status;
    out->stats = j->stats;
    out->t_submit = j->t_submit;
    out->t_start = j->t_start;
    out->t_end = j->t_end;
    out->slot = j->slot;
    sv->jobs.erase(it);
    delete j;
    if (sv->stop && sv->waiters == 0) sv->cv_idle.notify_all();
    return QCD_OK;
}

qcd_status qcd_server_info(qcd_server *sv, size_t *used_bytes, int *queued, int *running)
{
    if (!sv) return fail(QCD_ERR_INVALID_ARG, "server_info: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (used_bytes) *used_bytes = sv->used;
    if (queued) *queued = (int)sv->queue.size();
    if (running) {
        int r = 0;
        for (int b : sv->busy) r += b;
        *running = r;
    }
    return QCD_OK;
}

void qcd_server_destroy(qcd_server *sv)
{
    if (!sv) return;
    {
        // queued requests are cancelled; threads waiting for them return
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        const double t = sv->now();
        for (Job *j : sv->queue) {
            j->status = QCD_ERR_CANCELLED;
            j->t_start = j->t_end = t;
            j->done = true;
        }
        sv->queue.clear();
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
    }
    for (auto &t : sv->workers) t.join();  // running requests finish first
    {
        // no thread may still be inside qcd_server_wait when sv is freed
        std::unique_lock<std::mutex> lk(sv->mu);
        sv->cv_done.notify_all();
        sv->cv_idle.wait(lk, [&] { return sv->waiters == 0; });
    }
    cudaSetDevice(sv->device);
    for (auto &m : sv->slot_ctx)
        for (auto &kv : m) release(sv, kv.second);
    for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
    for (cudaStream_t s : sv->streams_lo) cudaStreamDestroy(s);
    for (auto &kv : sv->jobs) delete kv.second;
    delete sv;
}

}  // extern "C"
