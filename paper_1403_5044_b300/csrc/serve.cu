// The serving loop: solves of uneven meshes requested one at a time, run
// concurrently on one GPU.
//
// A request (mesh, F, eps) waits in a FIFO queue until a worker slot is free
// and its context fits the device-memory budget.  At admission the scheduler
// takes, besides the head of the queue, the later queued requests on the same
// mesh (up to max_group) and runs them as one batch context, so their
// residuals, Krylov steps and factorisations share launches.  Each admitted
// group runs on its own CUDA stream with its Newton/Krylov state resident in
// its context, so groups on different meshes overlap on the device: one
// group's latency-bound factorisation (a few SMs) runs beside another's
// residual kernels.  Admission is continuous: whenever a group finishes, its
// slot and memory go to the next requests in the queue.  Finished contexts
// may be kept and reused by later groups of the same shape (evicted least
// recently used when memory is needed).  Results (zeta on the mesh, the
// solver's counters, queue and run times) wait in the request's record until
// the caller polls for them.
//
// Every instance of a batch context runs the same kernel sequence, with the
// same launch plan, as it would alone, so a result does not depend on the
// mix it was served in.
#include "swj_internal.h"
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string.h>
#include <thread>
#include <vector>

namespace {

double wall_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

bool same_mesh(const swj_mesh &a, const swj_mesh &b)
{
    return a.N == b.N && a.M == b.M && a.x1 == b.x1 && a.dx == b.dx && a.dy == b.dy && a.n_rad == b.n_rad;
}

struct Request {
    long long id;
    swj_mesh mesh;
    double F, eps;
    bool done = false;
    int status = SWJ_PENDING;
    swj_stats st;
    std::vector<double> zeta;   // [M][N]
    double t_submit = 0, t_admit = 0, t_done = 0;
    int group = 0;
};

// A context held by the server (busy while a group runs in it).
struct Slot {
    swj_mesh mesh;
    int count = 0;
    size_t bytes = 0;          // footprint charged to the budget
    swj_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    double *u = nullptr, *z = nullptr;   // device: count unknown vectors, count zeta arrays
    double *zh = nullptr;                // pinned host copy of z
    bool busy = false;
    unsigned long long last_use = 0;
};

struct Job {
    std::vector<Request *> reqs;
    Slot *slot;
    bool fresh;                // the worker must create the context
};

}  // namespace

struct swj_server {
    swj_server_opts o;
    int dev = 0;
    size_t budget = 0;
    std::mutex m;
    std::condition_variable cv_sched, cv_work, cv_done;
    std::deque<Request *> queue;
    std::map<long long, Request *> reqs;
    std::vector<Slot *> slots;
    std::deque<Job> jobs;
    std::vector<std::thread> workers;
    std::thread sched;
    bool stop = false;
    long long next_id = 1;
    int active = 0;            // groups admitted and not finished
    size_t held = 0;           // bytes charged for slots (busy, idle or being created)
    unsigned long long tick = 0;
    swj_server_info info;
};

namespace {

void release_slot(Slot *s)
{
    if (s->ctx) swj_destroy(s->ctx);
    if (s->u) cudaFree(s->u);
    if (s->z) cudaFree(s->z);
    if (s->zh) cudaFreeHost(s->zh);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

int build_slot(swj_server *sv, Slot *s, const std::vector<Request *> &g)
{
    std::vector<double> F(g.size()), eps(g.size());
    for (size_t i = 0; i < g.size(); ++i) {
        F[i] = g[i]->F;
        eps[i] = g[i]->eps;
    }
    const size_t nu = 2 * (size_t)(s->mesh.N + 1) * s->mesh.M, nm = (size_t)s->mesh.N * s->mesh.M;
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return SWJ_ECUDA;
    int rc = swj_batch_create(&s->ctx, &s->mesh, s->count, F.data(), eps.data(), &sv->o.opts, s->stream);
    if (rc) return rc;
    if (cudaMalloc(&s->u, s->count * nu * sizeof(double)) != cudaSuccess) return SWJ_ENOMEM;
    if (cudaMalloc(&s->z, s->count * nm * sizeof(double)) != cudaSuccess) return SWJ_ENOMEM;
    if (cudaMallocHost(&s->zh, s->count * nm * sizeof(double)) != cudaSuccess) return SWJ_ENOMEM;
    return SWJ_OK;
}

// Solve one group in its slot; fills the requests' records (not yet marked done).
int run_group(swj_server *sv, Job &job)
{
    Slot *s = job.slot;
    const std::vector<Request *> &g = job.reqs;
    int rc = SWJ_OK;
    if (job.fresh) {
        rc = build_slot(sv, s, g);
    } else {
        std::vector<double> F(g.size()), eps(g.size());
        for (size_t i = 0; i < g.size(); ++i) {
            F[i] = g[i]->F;
            eps[i] = g[i]->eps;
        }
        rc = swj_batch_set_params(s->ctx, F.data(), eps.data());
    }
    if (rc) return rc;
    std::vector<swj_stats> st(g.size());
    rc = swj_initial_guess_flat(s->ctx, s->u);
    if (rc) return rc;
    int src = swj_solve(s->ctx, s->u, st.data());
    if (src == SWJ_ECUDA) return src;
    rc = swj_unpack(s->ctx, s->u, s->z, nullptr);
    if (rc) return rc;
    const size_t nm = (size_t)s->mesh.N * s->mesh.M;
    if (cudaMemcpyAsync(s->zh, s->z, g.size() * nm * sizeof(double), cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return SWJ_ECUDA;
    for (size_t i = 0; i < g.size(); ++i) {
        g[i]->st = st[i];
        g[i]->status = st[i].status;
        g[i]->zeta.assign(s->zh + i * nm, s->zh + (i + 1) * nm);
    }
    return SWJ_OK;
}

void worker_main(swj_server *sv)
{
    cudaSetDevice(sv->dev);
    for (;;) {
        Job job;
        {
            std::unique_lock<std::mutex> lk(sv->m);
            sv->cv_work.wait(lk, [&] { return sv->stop || !sv->jobs.empty(); });
            if (sv->jobs.empty()) return;   // stop with nothing left to run
            job = sv->jobs.front();
            sv->jobs.pop_front();
        }
        int rc = run_group(sv, job);
        const double t = wall_ms();
        Slot *drop = nullptr;
        {
            std::lock_guard<std::mutex> lk(sv->m);
            for (Request *r : job.reqs) {
                if (rc) r->status = rc;
                r->done = true;
                r->t_done = t;
                if (r->status == SWJ_OK) sv->info.completed++;
                else sv->info.failed++;
            }
            Slot *s = job.slot;
            s->busy = false;
            s->last_use = ++sv->tick;
            if (rc || !sv->o.keep_contexts) {
                // a slot that failed (or is not kept) gives its memory back
                for (size_t i = 0; i < sv->slots.size(); ++i)
                    if (sv->slots[i] == s) {
                        sv->slots.erase(sv->slots.begin() + i);
                        break;
                    }
                sv->held -= s->bytes;
                drop = s;
            }
            sv->active--;
        }
        if (drop) release_slot(drop);
        sv->cv_sched.notify_all();
        sv->cv_done.notify_all();
    }
}

// Called with the lock held.  Picks the group at the head of the queue and a
// slot for it; returns false when nothing can be admitted now.  Idle slots to
// evict are moved to `evict` (released by the caller without the lock).
// Group sizes are powers of two, so that kept contexts are reused often.
bool admit(swj_server *sv, std::vector<Slot *> &evict)
{
    if (sv->queue.empty() || sv->active >= sv->o.max_active) return false;
    Request *head = sv->queue.front();
    std::vector<size_t> idx{0};
    for (size_t i = 1; i < sv->queue.size() && (int)idx.size() < sv->o.max_group; ++i)
        if (same_mesh(sv->queue[i]->mesh, head->mesh)) idx.push_back(i);
    int g = 1;
    while (2 * g <= (int)idx.size()) g *= 2;
    size_t idle = 0;
    for (Slot *s : sv->slots)
        if (!s->busy) idle += s->bytes;
    Slot *use = nullptr;
    bool fresh = false;
    for (; g >= 1 && !use; g /= 2) {
        for (Slot *s : sv->slots)
            if (!s->busy && s->count == g && same_mesh(s->mesh, head->mesh)) {
                use = s;
                break;
            }
        if (use) {
            sv->info.contexts_reused++;
            break;
        }
        size_t need = swj_footprint_bytes(&head->mesh, g, &sv->o.opts);
        if (!need) continue;
        need += (size_t)g * (2 * (size_t)(head->mesh.N + 1) * head->mesh.M +
                             (size_t)head->mesh.N * head->mesh.M) * sizeof(double);   // u and zeta
        if (sv->held - idle + need > sv->budget) continue;
        // a new context; evict least recently used idle slots until it fits
        while (sv->held + need > sv->budget) {
            Slot *lru = nullptr;
            for (Slot *s : sv->slots)
                if (!s->busy && (!lru || s->last_use < lru->last_use)) lru = s;
            if (!lru) break;
            for (size_t i = 0; i < sv->slots.size(); ++i)
                if (sv->slots[i] == lru) {
                    sv->slots.erase(sv->slots.begin() + i);
                    break;
                }
            sv->held -= lru->bytes;
            sv->info.contexts_evicted++;
            evict.push_back(lru);
        }
        use = new Slot();
        use->mesh = head->mesh;
        use->count = g;
        use->bytes = need;
        sv->slots.push_back(use);
        sv->held += need;
        fresh = true;
        sv->info.contexts_created++;
        break;
    }
    if (!use) return false;   // wait for busy slots to finish
    idx.resize(use->count);
    use->busy = true;
    Job job;
    job.slot = use;
    job.fresh = fresh;
    const double t = wall_ms();
    for (size_t k = idx.size(); k-- > 0;) {
        Request *r = sv->queue[idx[k]];
        r->t_admit = t;
        r->group = (int)idx.size();
        job.reqs.insert(job.reqs.begin(), r);
        sv->queue.erase(sv->queue.begin() + idx[k]);
    }
    sv->active++;
    if (sv->active > sv->info.peak_active) sv->info.peak_active = sv->active;
    if (sv->held > sv->info.peak_bytes_held) sv->info.peak_bytes_held = sv->held;
    sv->jobs.push_back(job);
    return true;
}

void sched_main(swj_server *sv)
{
    cudaSetDevice(sv->dev);
    std::unique_lock<std::mutex> lk(sv->m);
    while (!sv->stop) {
        std::vector<Slot *> evict;
        bool any = false;
        while (admit(sv, evict)) any = true;
        if (!evict.empty()) {
            lk.unlock();
            for (Slot *s : evict) release_slot(s);
            lk.lock();
        }
        if (any) {
            sv->cv_work.notify_all();
            continue;
        }
        sv->cv_sched.wait(lk);
    }
}

}  // namespace

extern "C" {

void swj_server_default_opts(swj_server_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->hbm_budget_bytes = 0;
    o->max_active = 4;
    o->max_group = 8;
    o->keep_contexts = 1;
    swj_default_opts(&o->opts);
}

int swj_server_create(swj_server **out, const swj_server_opts *opts)
{
    if (!out) return SWJ_EINVAL;
    *out = nullptr;
    swj_server_opts o;
    if (opts) o = *opts; else swj_server_default_opts(&o);
    if (o.max_active < 1 || o.max_active > 256 || o.max_group < 1 || o.max_group > 1024) return SWJ_EINVAL;
    swj_mesh tiny = {4, 3, -1.0, 0.5, 0.5, 0.05};
    if (swj_footprint_bytes(&tiny, 1, &o.opts) == 0) return SWJ_EINVAL;   // checks the options
    swj_server *sv = new (std::nothrow) swj_server();
    if (!sv) return SWJ_ENOMEM;
    sv->o = o;
    memset(&sv->info, 0, sizeof(sv->info));
    size_t fr = 0, tot = 0;
    if (cudaGetDevice(&sv->dev) != cudaSuccess || cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        delete sv;
        return SWJ_ECUDA;
    }
    sv->budget = o.hbm_budget_bytes ? o.hbm_budget_bytes : (size_t)(0.8 * (double)fr);
    sv->sched = std::thread(sched_main, sv);
    for (int i = 0; i < o.max_active; ++i) sv->workers.emplace_back(worker_main, sv);
    *out = sv;
    return SWJ_OK;
}

int swj_server_submit(swj_server *sv, const swj_mesh *mesh, double F, double eps, long long *id)
{
    if (!sv || !mesh || !id) return SWJ_EINVAL;
    if (!(F > 0.0) || !(eps >= 0.0)) return SWJ_EINVAL;
    size_t need = swj_footprint_bytes(mesh, 1, &sv->o.opts);
    if (!need) return SWJ_EINVAL;
    if (need > sv->budget) return SWJ_ENOMEM;   // could never be admitted
    Request *r = new (std::nothrow) Request();
    if (!r) return SWJ_ENOMEM;
    r->mesh = *mesh;
    r->F = F;
    r->eps = eps;
    memset(&r->st, 0, sizeof(r->st));
    {
        std::lock_guard<std::mutex> lk(sv->m);
        r->id = sv->next_id++;
        r->t_submit = wall_ms();
        sv->reqs[r->id] = r;
        sv->queue.push_back(r);
        sv->info.submitted++;
        *id = r->id;
    }
    sv->cv_sched.notify_all();
    return SWJ_OK;
}

int swj_server_poll(swj_server *sv, long long id, int wait, swj_stats *st, double *zeta,
                    swj_request_times *times)
{
    if (!sv) return SWJ_EINVAL;
    Request *r = nullptr;
    {
        std::unique_lock<std::mutex> lk(sv->m);
        auto it = sv->reqs.find(id);
        if (it == sv->reqs.end()) return SWJ_EINVAL;
        r = it->second;
        if (!r->done) {
            if (!wait) return SWJ_PENDING;
            sv->cv_done.wait(lk, [&] { return r->done; });
        }
        sv->reqs.erase(id);
    }
    if (st) *st = r->st;
    if (zeta && !r->zeta.empty()) memcpy(zeta, r->zeta.data(), r->zeta.size() * sizeof(double));
    if (times) {
        times->queue_ms = r->t_admit - r->t_submit;
        times->run_ms = r->t_done - r->t_admit;
        times->latency_ms = r->t_done - r->t_submit;
        times->group_size = r->group;
    }
    int status = r->status;
    delete r;
    return status;
}

int swj_server_get_info(swj_server *sv, swj_server_info *info)
{
    if (!sv || !info) return SWJ_EINVAL;
    std::lock_guard<std::mutex> lk(sv->m);
    *info = sv->info;
    info->queued = (int)sv->queue.size();
    info->active = sv->active;
    info->bytes_held = sv->held;
    info->budget_bytes = sv->budget;
    return SWJ_OK;
}

int swj_server_drain(swj_server *sv)
{
    if (!sv) return SWJ_EINVAL;
    std::unique_lock<std::mutex> lk(sv->m);
    sv->cv_done.wait(lk, [&] { return sv->queue.empty() && sv->active == 0; });
    return SWJ_OK;
}

void swj_server_destroy(swj_server *sv)
{
    if (!sv) return;
    {
        std::unique_lock<std::mutex> lk(sv->m);
        // queued requests are dropped; admitted groups finish first
        for (Request *r : sv->queue) {
            sv->reqs.erase(r->id);
            delete r;
        }
        sv->queue.clear();
        sv->cv_done.wait(lk, [&] { return sv->active == 0; });
        sv->stop = true;
    }
    sv->cv_sched.notify_all();
    sv->cv_work.notify_all();
    if (sv->sched.joinable()) sv->sched.join();
    for (std::thread &t : sv->workers)
        if (t.joinable()) t.join();
    cudaSetDevice(sv->dev);
    for (Slot *s : sv->slots) release_slot(s);
    for (auto &kv : sv->reqs) delete kv.second;
    delete sv;
}

}  // extern "C"
