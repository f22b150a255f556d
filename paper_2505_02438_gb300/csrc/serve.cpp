// Continuous-batching request server (include/soptx_serve.h).
//
// One scheduler thread owns admission and completion: it polls the completion
// events of the requests in flight, then admits queued requests in arrival
// order while a slot is free and the job's mesh is resident or fits under the
// HBM cap (evicting meshes of idle jobs, least recently used first).  Mesh
// setup runs with the server lock released, so submitters and waiters are
// never blocked behind it.  Requests of one job share that job's stream, so
// they run in order and never overlap on the mesh's scratch; different jobs
// run on different streams of the pool and overlap on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <sys/prctl.h>

#include "internal.h"
#include "../../include/soptx_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

double us_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::micro>(b - a).count();
}

struct Job {
    uint64_t id = 0;
    soptx_mesh mesh = nullptr;
    int64_t bytes = 0;
    int in_flight = 0;
    uint64_t last_use = 0;
    int stream = 0;
    int64_t nnz = 0;
    int64_t known_bytes = 0;   // device bytes of this job's mesh once it has been built
    int64_t bound_bytes = 0;   // mesh_bytes_bound of its request, before it has been built
};

struct Req {
    uint64_t ticket = 0;
    soptx_request r{};
    Clock::time_point t_submit, t_admit;
    soptx_result res{};
    bool done = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    Job *job = nullptr;
};

// The most cells at one vertex of a request's mesh: a bound on the cells that
// any two of its nodes share (those cells all hold a vertex of the first node's
// edge, face or cell).  Ids out of range are skipped (mesh creation rejects them).
int64_t max_cells_at_vertex(const soptx_request &r, int nv)
{
    if (!r.cell_vertices || r.n_cells <= 0) return 0;
    std::vector<int32_t> cnt((size_t)r.n_vertices, 0);
    int32_t best = 0;
    for (int64_t q = 0; q < r.n_cells * nv; q++) {
        const int32_t v = r.cell_vertices[q];
        if (v >= 0 && v < r.n_vertices) best = std::max(best, ++cnt[(size_t)v]);
    }
    return best;
}

// Upper bound of a mesh's device bytes from its input alone (every array of
// soptx_mesh_create at its largest), used before the mesh exists.  The node-pair
// tables of the pair kernel hold R records (a pair and one cell of it: at most
// nb (nb + 1) / 2 per cell in 2D, nb^2 in 3D) padded per tile of 32 pairs to its
// largest count; within a window of pairs sorted by count a tile's largest is at
// most the previous tile's smallest, so a window pads at most 32 times its
// largest count (at most the most cells at a vertex, c) above its own records,
// and windows hold 4096 pairs or more but the last.  In 2D with FP64 element
// matrices each record also carries its 2 x 2 block (32 bytes).
int64_t mesh_bytes_bound(const soptx_request &r)
{
    static const int nb_tab[4][4] = {{0, 3, 6, 10}, {0, 4, 10, 20}, {0, 4, 9, 16}, {0, 8, 27, 64}};
    static const int nv_tab[4] = {3, 4, 4, 8};
    const int64_t nb = nb_tab[r.cell][std::min(std::max(r.order, 1), 3)];
    const int64_t ldof = r.dim * nb, nc = r.n_cells;
    const int64_t ee = nc * ldof * ldof;          // >= nnz
    const int64_t nn = r.n_vertices + nc * nb;    // >= nodes
    const int64_t base = ee * 8 /* K_e (cached) */ + ee * 4 /* indices */ + nc * nb * nb * 2 /* pos */ +
                         nc * nb * (4 + 4 + 4 + 1 + 8) /* cell_node, inc, inc_e, inc_a, partials */ +
                         nn * r.dim * (8 + 8) + nn * 20 + nc * 120 + (1 << 20);
    const int64_t c = std::min<int64_t>(max_cells_at_vertex(r, nv_tab[r.cell]), 1023);
    const int64_t rec = nc * (r.dim == 2 ? nb * (nb + 1) / 2 : nb * nb);
    const int64_t windows = rec / 4096 + 1;
    const int64_t padded = rec + windows * 32 * c;
    const int64_t lanes = rec + windows * 32 + 7 * 32;   // and the last chunk of 8 tiles filled
    const int64_t per_rec = 4 + 2 + (r.dim == 2 && r.prec == SOPTX_ELEM_FP64 ? 32 : 0);
    return base + padded * per_rec + lanes * 12 + (lanes / 32 + 32) * 4 + 64;
}

}  // namespace

struct soptx_server_s {
    soptx_server_opts opts{};
    std::vector<cudaStream_t> streams;
    cudaStream_t gstream = nullptr;   // the grouped launches of small lattice requests
    std::vector<Req *> group;         // requests gathered in this scheduler pass
    cudaEvent_t t0 = nullptr;   // origin of the requests' device timeline
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Req *> queue;
    std::vector<Req *> inflight;
    std::unordered_map<uint64_t, Req *> tickets;
    std::unordered_map<uint64_t, Job *> jobs;
    int64_t resident = 0;
    soptx_server_stats stats{};
    uint64_t next_ticket = 1, use_clock = 0;
    int next_stream = 0;
    bool stop = false;
    bool setup_in_progress = false;
    std::thread th;

    void finish(Req *q, soptx_status st)
    {
        q->res.status = st;
        q->res.latency_us = us_between(q->t_submit, Clock::now());
        q->done = true;
        if (st == SOPTX_OK) stats.completed++;
        else stats.failed++;
        cv_done.notify_all();
    }

    void poll_completions()
    {
        for (size_t k = 0; k < inflight.size();) {
            Req *q = inflight[k];
            cudaError_t e = cudaEventQuery(q->ev1);
            if (e == cudaErrorNotReady) {
                k++;
                continue;
            }
            float ms = 0.f, ms0 = 0.f, ms1 = 0.f;
            if (e == cudaSuccess) {
                cudaEventElapsedTime(&ms, q->ev0, q->ev1);
                if (cudaEventElapsedTime(&ms0, t0, q->ev0) != cudaSuccess ||
                    cudaEventElapsedTime(&ms1, t0, q->ev1) != cudaSuccess) {
                    cudaGetLastError();
                    ms0 = ms1 = 0.f;
                }
            } else {
                cudaGetLastError();
            }
            q->res.gpu_us = 1e3 * ms;
            q->res.gpu_start_us = 1e3 * ms0;
            q->res.gpu_end_us = 1e3 * ms1;
            q->job->in_flight--;
            finish(q, e == cudaSuccess ? SOPTX_OK : SOPTX_ECUDA);
            inflight.erase(inflight.begin() + k);
        }
    }

    // Evicts idle meshes (LRU first) until `need` more bytes fit; true on success.
    bool make_room(int64_t need)
    {
        while (resident + need > opts.hbm_cap_bytes) {
            Job *victim = nullptr;
            for (auto &kv : jobs)
                if (kv.second->mesh && kv.second->in_flight == 0 &&
                    (!victim || kv.second->last_use < victim->last_use))
                    victim = kv.second;
            if (!victim) return false;
            soptx_mesh_destroy(victim->mesh);
            victim->mesh = nullptr;
            resident -= victim->bytes;
            victim->bytes = 0;
            stats.evictions++;
        }
        return true;
    }

    soptx_status launch(Req *q)
    {
        Job *j = q->job;
        cudaStream_t st = streams[j->stream];
        q->t_admit = Clock::now();
        q->res.queue_us = us_between(q->t_submit, q->t_admit);
        q->res.nnz = j->nnz;
        if (cudaEventCreate(&q->ev0) != cudaSuccess || cudaEventCreate(&q->ev1) != cudaSuccess) {
            cudaGetLastError();
            return SOPTX_ECUDA;
        }
        cudaEventRecord(q->ev0, st);
        soptx_status s = q->r.d_vals
                             ? soptx_assemble_and_sensitivity(j->mesh, q->r.d_rho, q->r.d_u, q->r.d_vals, q->r.d_dc,
                                                              q->r.d_c, st)
                             : soptx_sensitivity(j->mesh, q->r.d_rho, q->r.d_u, q->r.d_dc, q->r.d_c, st);
        if (s != SOPTX_OK) return s;
        if (cudaEventRecord(q->ev1, st) != cudaSuccess) {
            cudaGetLastError();
            return SOPTX_ECUDA;
        }
        j->in_flight++;
        j->last_use = ++use_clock;
        inflight.push_back(q);
        return SOPTX_OK;
    }

    // A request whose job mesh takes the grouped kernel: 1 = gathered into this
    // pass's group, 0 = not such a request, -1 = its job still has one in flight
    // (it stays queued, so the job's requests run in order).
    int try_group(Req *q)
    {
        Job *j = q->job;
        if (!opts.group_small || !q->r.d_vals || !soptx::lattice_groupable(*j->mesh)) return 0;
        if (j->in_flight > 0) return -1;
        q->t_admit = Clock::now();
        q->res.queue_us = us_between(q->t_submit, q->t_admit);
        q->res.nnz = j->nnz;
        // counted in flight from now on: its mesh is not evicted while the group is gathered
        j->in_flight++;
        j->last_use = ++use_clock;
        group.push_back(q);
        return 1;
    }

    // One launch for the gathered requests; each gets events at the group's start
    // and end on the group stream.
    void flush_group()
    {
        if (group.empty()) return;
        const int n = (int)group.size();
        std::vector<soptx_mesh> ms(n);
        std::vector<const double *> rho(n), u(n);
        std::vector<double *> vals(n), dc(n), c(n);
        soptx_status s = SOPTX_OK;
        for (int k = 0; k < n; k++) {
            Req *q = group[k];
            ms[k] = q->job->mesh;
            rho[k] = q->r.d_rho;
            u[k] = q->r.d_u;
            vals[k] = q->r.d_vals;
            dc[k] = q->r.d_dc;
            c[k] = q->r.d_c;
            if (s == SOPTX_OK && (cudaEventCreate(&q->ev0) != cudaSuccess || cudaEventCreate(&q->ev1) != cudaSuccess ||
                                  cudaEventRecord(q->ev0, gstream) != cudaSuccess)) {
                cudaGetLastError();
                s = SOPTX_ECUDA;
            }
        }
        if (s == SOPTX_OK)
            s = soptx_assemble_and_sensitivity_group(n, ms.data(), rho.data(), u.data(), vals.data(), dc.data(),
                                                     c.data(), gstream);
        for (int k = 0; k < n && s == SOPTX_OK; k++)
            if (cudaEventRecord(group[k]->ev1, gstream) != cudaSuccess) {
                cudaGetLastError();
                s = SOPTX_ECUDA;
            }
        for (Req *q : group) {
            if (s != SOPTX_OK) {
                q->job->in_flight--;
                finish(q, s);
                continue;
            }
            inflight.push_back(q);
        }
        stats.groups += s == SOPTX_OK ? 1 : 0;
        group.clear();
    }

    void run()
    {
        // the completion polls sleep 10 us; with the kernel's default timer slack
        // (50 us) such a sleep lasts about 60 us, with 1 us of slack about 11 us
        prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
        cudaSetDevice(opts.device);
        std::unique_lock<std::mutex> lock(mu);
        for (;;) {
            poll_completions();
            if (stop && queue.empty() && inflight.empty()) break;
            // admissions in arrival order; a request that does not fit yet is skipped
            bool progressed = false;
            for (auto it = queue.begin(); it != queue.end() && (int)(inflight.size() + group.size()) < opts.max_slots;) {
                Req *q = *it;
                if (stop) {
                    finish(q, SOPTX_EBUSY);
                    it = queue.erase(it);
                    continue;
                }
                Job *&jp = jobs[q->r.job];
                if (!jp) {
                    jp = new Job();
                    jp->id = q->r.job;
                    jp->stream = next_stream++ % (int)streams.size();
                }
                Job *j = jp;
                q->job = j;
                if (!j->mesh) {
                    if (!j->known_bytes && !j->bound_bytes) j->bound_bytes = mesh_bytes_bound(q->r);
                    const int64_t bound = j->known_bytes ? j->known_bytes : j->bound_bytes;
                    const bool fits = make_room(std::min(bound, opts.hbm_cap_bytes - 0));
                    if (!fits && resident > 0) {   // wait for jobs in flight to go idle
                        ++it;
                        continue;
                    }
                    // set the mesh up with the lock released
                    setup_in_progress = true;
                    soptx_request rq = q->r;
                    cudaStream_t st = streams[j->stream];
                    lock.unlock();
                    soptx_mesh m = nullptr;
                    soptx_status s = soptx_mesh_create(rq.dim, rq.cell, rq.order, rq.n_vertices, rq.coords,
                                                       rq.n_cells, rq.cell_vertices, &rq.mat, rq.prec, st, &m);
                    int64_t bytes = 0, nnz = 0;
                    if (s == SOPTX_OK) {
                        soptx_mesh_device_bytes(m, &bytes);
                        soptx_mesh_info(m, nullptr, &nnz, nullptr, nullptr);
                    }
                    lock.lock();
                    if (s == SOPTX_OK) j->known_bytes = bytes;
                    setup_in_progress = false;
                    stats.mesh_setups++;
                    if (s == SOPTX_OK && resident + bytes > opts.hbm_cap_bytes && !make_room(bytes)) {
                        soptx_mesh_destroy(m);
                        m = nullptr;
                        s = (resident == 0) ? SOPTX_ENOMEM : SOPTX_EBUSY;
                        if (s == SOPTX_EBUSY) {   // retry once others go idle
                            it = queue.begin();
                            progressed = true;
                            break;
                        }
                    }
                    if (s != SOPTX_OK) {
                        finish(q, s);
                        queue.erase(std::find(queue.begin(), queue.end(), q));
                        it = queue.begin();
                        progressed = true;
                        continue;
                    }
                    j->mesh = m;
                    j->bytes = bytes;
                    j->nnz = nnz;
                    resident += bytes;
                    stats.peak_resident_bytes = std::max(stats.peak_resident_bytes, resident);
                    q->res.mesh_was_resident = 0;
                    // the queue may have changed while unlocked: restart the scan
                    const int gr = try_group(q);
                    if (gr >= 0) {
                        auto pos = std::find(queue.begin(), queue.end(), q);
                        queue.erase(pos);
                        if (gr == 0) {
                            soptx_status ls = launch(q);
                            if (ls != SOPTX_OK) {
                                j->in_flight = std::max(0, j->in_flight);
                                finish(q, ls);
                            }
                        }
                    }
                    it = queue.begin();
                    progressed = true;
                    continue;
                }
                q->res.mesh_was_resident = 1;
                const int gr = try_group(q);
                if (gr < 0) {
                    ++it;
                    continue;
                }
                if (gr == 0) {
                    soptx_status ls = launch(q);
                    if (ls != SOPTX_OK) finish(q, ls);
                }
                it = queue.erase(it);
                progressed = true;
            }
            flush_group();
            if (progressed) continue;
            if (!inflight.empty()) {
                lock.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(10));
                lock.lock();
            } else {
                cv_sched.wait(lock, [&] { return stop || !queue.empty(); });
                if (stop && queue.empty() && inflight.empty()) break;
            }
        }
    }
};

extern "C" {

soptx_status soptx_server_create(const soptx_server_opts *opts, soptx_server *out)
{
    if (!opts || !out) SOPTX_FAIL(SOPTX_EINVAL, "opts / out is NULL");
    *out = nullptr;
    if (opts->hbm_cap_bytes <= 0 || opts->max_slots < 1 || opts->n_streams < 1 || opts->max_queue < 1)
        SOPTX_FAIL(SOPTX_EINVAL, "need hbm_cap_bytes > 0, max_slots >= 1, n_streams >= 1, max_queue >= 1");
    soptx_server_s *s = new (std::nothrow) soptx_server_s();
    if (!s) SOPTX_FAIL(SOPTX_ENOMEM, "host allocation failed");
    s->opts = *opts;
    if (cudaSetDevice(opts->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        SOPTX_FAIL(SOPTX_ECUDA, "cudaSetDevice failed");
    }
    for (int k = 0; k < opts->n_streams; k++) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto x : s->streams) cudaStreamDestroy(x);
            delete s;
            SOPTX_FAIL(SOPTX_ECUDA, "cudaStreamCreate failed");
        }
        s->streams.push_back(st);
    }
    if (cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&s->t0) != cudaSuccess || cudaEventRecord(s->t0, s->streams[0]) != cudaSuccess ||
        cudaEventSynchronize(s->t0) != cudaSuccess) {
        cudaGetLastError();
        if (s->t0) cudaEventDestroy(s->t0);
        if (s->gstream) cudaStreamDestroy(s->gstream);
        for (auto x : s->streams) cudaStreamDestroy(x);
        delete s;
        SOPTX_FAIL(SOPTX_ECUDA, "timeline event");
    }
    s->th = std::thread([s] { s->run(); });
    *out = s;
    return SOPTX_OK;
}

soptx_status soptx_serve_submit(soptx_server s, const soptx_request *r, uint64_t *ticket)
{
    if (!s || !r || !ticket) SOPTX_FAIL(SOPTX_EINVAL, "server / request / ticket is NULL");
    if (r->dim < 2 || r->dim > 3 || (int)r->cell < SOPTX_TRI || (int)r->cell > SOPTX_HEX || r->order < 1 ||
        r->order > 3 || r->n_cells < 0 || r->n_vertices < 1 || !r->coords || (r->n_cells > 0 && !r->cell_vertices))
        SOPTX_FAIL(SOPTX_EINVAL, "malformed mesh description in the request");
    if (r->n_cells > 0 && (!r->d_rho || !r->d_u || !r->d_dc)) SOPTX_FAIL(SOPTX_EINVAL, "d_rho / d_u / d_dc is NULL");
    Req *q = new (std::nothrow) Req();
    if (!q) SOPTX_FAIL(SOPTX_ENOMEM, "host allocation failed");
    q->r = *r;
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) {
            delete q;
            SOPTX_FAIL(SOPTX_EBUSY, "server is shutting down");
        }
        if ((int)s->queue.size() >= s->opts.max_queue) {
            delete q;
            SOPTX_FAIL(SOPTX_EBUSY, "request queue is full");
        }
        q->ticket = s->next_ticket++;
        s->tickets[q->ticket] = q;
        s->queue.push_back(q);
        s->stats.submitted++;
    }
    s->cv_sched.notify_one();
    *ticket = q->ticket;
    return SOPTX_OK;
}

soptx_status soptx_serve_mesh_bytes_bound(const soptx_request *r, int64_t *bytes)
{
    if (!r || !bytes) SOPTX_FAIL(SOPTX_EINVAL, "request / bytes is NULL");
    if (r->dim < 2 || r->dim > 3 || (int)r->cell < SOPTX_TRI || (int)r->cell > SOPTX_HEX || r->order < 1 ||
        r->order > 3 || r->n_cells < 0 || r->n_vertices < 1 || !r->coords || (r->n_cells > 0 && !r->cell_vertices))
        SOPTX_FAIL(SOPTX_EINVAL, "malformed mesh description in the request");
    try {
        *bytes = mesh_bytes_bound(*r);
    } catch (const std::bad_alloc &) {
        SOPTX_FAIL(SOPTX_ENOMEM, "host allocation failed");
    }
    return SOPTX_OK;
}

soptx_status soptx_serve_poll(soptx_server s, uint64_t ticket, int32_t *done)
{
    if (!s || !done) SOPTX_FAIL(SOPTX_EINVAL, "server / done is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) SOPTX_FAIL(SOPTX_ENOTFOUND, "unknown ticket");
    *done = it->second->done ? 1 : 0;
    return SOPTX_OK;
}

soptx_status soptx_serve_wait(soptx_server s, uint64_t ticket, int64_t timeout_us, soptx_result *res)
{
    if (!s || !res) SOPTX_FAIL(SOPTX_EINVAL, "server / result is NULL");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) SOPTX_FAIL(SOPTX_ENOTFOUND, "unknown or already collected ticket");
    Req *q = it->second;
    if (timeout_us < 0) {
        s->cv_done.wait(lock, [&] { return q->done; });
    } else if (!s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), [&] { return q->done; })) {
        SOPTX_FAIL(SOPTX_ETIMEOUT, "request not finished within the timeout");
    }
    *res = q->res;
    s->tickets.erase(it);
    if (q->ev0) cudaEventDestroy(q->ev0);
    if (q->ev1) cudaEventDestroy(q->ev1);
    delete q;
    return SOPTX_OK;
}

soptx_status soptx_server_stats_get(soptx_server s, soptx_server_stats *out)
{
    if (!s || !out) SOPTX_FAIL(SOPTX_EINVAL, "server / stats is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    out->resident_bytes = s->resident;
    out->in_flight = (int32_t)s->inflight.size();
    out->queued = (int32_t)s->queue.size();
    int32_t nres = 0;
    for (auto &kv : s->jobs)
        if (kv.second->mesh) nres++;
    out->resident_meshes = nres;
    return SOPTX_OK;
}

soptx_status soptx_server_destroy(soptx_server s)
{
    if (!s) return SOPTX_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto &kv : s->tickets) {
        if (kv.second->ev0) cudaEventDestroy(kv.second->ev0);
        if (kv.second->ev1) cudaEventDestroy(kv.second->ev1);
        delete kv.second;
    }
    for (auto &kv : s->jobs) {
        if (kv.second->mesh) soptx_mesh_destroy(kv.second->mesh);
        delete kv.second;
    }
    for (auto st : s->streams) cudaStreamDestroy(st);
    if (s->gstream) cudaStreamDestroy(s->gstream);
    if (s->t0) cudaEventDestroy(s->t0);
    delete s;
    return SOPTX_OK;
}

}  // extern "C"
