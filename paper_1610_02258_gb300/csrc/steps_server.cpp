// Served form: continuous batching of simulation jobs on one GPU.
//
// Host-side scheduling on top of the C ABI: jobs are clones of a prototype
// simulation (steps_sim_clone), admitted first come first served while a slot
// is free and their device memory fits the budget, and advanced together in
// rounds. A round is one batched run per group of running jobs that moves
// every job by up to wave_windows windows of its own tau, stopping on its
// window grid or at its t_end, so no extra shortened windows are inserted.
// With the generic kernel all running jobs form one group; otherwise jobs
// are grouped by model structure, each group runs the step kernel compiled
// for its model, and the groups' batches run at the same time on streams of
// their own. Finished jobs leave between rounds (counts copied to the host,
// device memory freed); a group's batch is re-formed only when its set of
// running jobs changed. Every draw is addressed by (job seed, window, tet),
// so a job's result does not depend on what runs beside it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "steps_internal.h"

namespace {

struct Job {
    const steps_sim *proto = nullptr;
    uint64_t seed = 0;
    double t_end = 0.0;
    int32_t state = 0;             // 0 queued, 1 running, 2 finished, 3 result taken
    std::vector<int32_t> counts;   // initial counts until admitted, final counts once finished
    steps_sim *sim = nullptr;      // while running
    int64_t bytes = 0;             // device bytes while running
    uint64_t windows = 0;
    double t = 0.0;
};

// Running jobs that advance in one batched launch per window.
struct Group {
    std::string key;               // model structure ("" = every job, generic kernel)
    std::vector<int64_t> running;  // job ids, in batch member order
    steps_batch *batch = nullptr;  // over `running` when valid
    bool valid = false;
    cudaStream_t stream = nullptr; // the server's stream (one group) or one of the group's own
    bool own_stream = false;
    bool enqueued = false;
};

}  // namespace

struct steps_server {
    steps_server_options opt{};
    void *stream = nullptr;
    std::vector<Job> jobs;
    std::deque<int64_t> queue;     // queued job ids, by submission
    std::vector<Group> groups;
    std::vector<int> job_group;    // group index of every job
    int32_t n_running = 0;
    uint64_t rounds = 0, rebuilds = 0, launches = 0;
    int64_t bytes_running = 0;

    void drop_batch(Group &g) {
        if (g.batch) {
            uint64_t l = 0;
            if (steps_batch_info(g.batch, nullptr, &l, nullptr) == STEPS_OK) launches += l;
            steps_batch_destroy(g.batch);
        }
        g.batch = nullptr;
        g.valid = false;
    }

    ~steps_server() {
        for (Group &g : groups) {
            drop_batch(g);
            if (g.own_stream) cudaStreamDestroy(g.stream);
        }
        for (Job &j : jobs)
            if (j.sim) steps_sim_destroy(j.sim);
    }
};

namespace {

bool valid_job(const steps_server *srv, int64_t job) { return job >= 0 && job < (int64_t)srv->jobs.size(); }

// The group a job of this prototype runs in (created on first use).
int group_of(steps_server *srv, const steps_sim *proto, int *out) {
    const std::string key = srv->opt.specialize < 0 ? std::string() : steps::sim_structure_key(proto);
    for (size_t g = 0; g < srv->groups.size(); ++g)
        if (srv->groups[g].key == key) {
            *out = (int)g;
            return STEPS_OK;
        }
    Group g;
    g.key = key;
    if (srv->opt.specialize < 0) {
        g.stream = (cudaStream_t)srv->stream;
    } else {
        if (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            steps::set_error("steps_server_submit: cudaStreamCreateWithFlags failed");
            return STEPS_ERR_CUDA;
        }
        g.own_stream = true;
    }
    try {
        srv->groups.push_back(g);
    } catch (const std::bad_alloc &) {
        if (g.own_stream) cudaStreamDestroy(g.stream);
        steps::set_error("steps_server_submit: out of host memory");
        return STEPS_ERR_OOM;
    }
    *out = (int)srv->groups.size() - 1;
    return STEPS_OK;
}

// Clone the prototype, set its counts: the job is running.
int admit(steps_server *srv, int64_t id) {
    Job &j = srv->jobs[(size_t)id];
    steps_sim *s = nullptr;
    int rc = steps_sim_clone(j.proto, j.seed, srv->stream, &s);
    if (rc) return rc;
    rc = steps_set_counts_all(s, j.counts.data());
    if (rc == STEPS_OK) rc = steps_sim_device_bytes(s, &j.bytes);
    if (rc) {
        steps_sim_destroy(s);
        return rc;
    }
    j.sim = s;
    j.state = 1;
    j.counts.clear();
    j.counts.shrink_to_fit();
    Group &g = srv->groups[(size_t)srv->job_group[(size_t)id]];
    g.running.push_back(id);
    g.valid = false;
    srv->n_running += 1;
    srv->bytes_running += j.bytes;
    return STEPS_OK;
}

// Reached t_end: final counts to the host, device memory freed.
int retire(steps_server *srv, int64_t id) {
    Job &j = srv->jobs[(size_t)id];
    int64_t nt = 0;
    int32_t ns = 0;
    int rc = steps_sim_shape(j.sim, &nt, &ns);
    if (rc) return rc;
    try {
        j.counts.assign((size_t)ns * (size_t)nt, 0);
    } catch (const std::bad_alloc &) {
        steps::set_error("steps_server_step: out of host memory for a job's result");
        return STEPS_ERR_OOM;
    }
    rc = steps_get_counts_all(j.sim, j.counts.data());
    if (rc) return rc;
    steps_get_windows(j.sim, &j.windows, nullptr);
    steps_get_time(j.sim, &j.t);
    steps_sim_destroy(j.sim);
    j.sim = nullptr;
    j.state = 2;
    srv->bytes_running -= j.bytes;
    srv->n_running -= 1;
    j.bytes = 0;
    return STEPS_OK;
}

}  // namespace

extern "C" {

void steps_server_options_default(steps_server_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->device_budget = 0;
    opt->max_jobs = 64;
    opt->wave_windows = 16;
    opt->block = 256;
    opt->specialize = -1;
}

int steps_server_create(const steps_server_options *opt, void *cuda_stream, steps_server **out) {
    if (!out) {
        steps::set_error("steps_server_create: NULL argument");
        return STEPS_ERR_ARG;
    }
    *out = nullptr;
    steps_server_options o;
    steps_server_options_default(&o);
    if (opt) o = *opt;
    if (o.block == 0) o.block = 256;
    if (o.max_jobs < 1 || o.wave_windows < 1 || o.device_budget < 0 ||
        (o.block != 64 && o.block != 128 && o.block != 256 && o.block != 512) || o.specialize < -1 ||
        o.specialize > 1) {
        steps::set_error("steps_server_create: need max_jobs >= 1, wave_windows >= 1, device_budget >= 0, "
                         "block 64/128/256/512, specialize -1/0/1");
        return STEPS_ERR_ARG;
    }
    steps_server *s = new (std::nothrow) steps_server;
    if (!s) {
        steps::set_error("steps_server_create: out of host memory");
        return STEPS_ERR_OOM;
    }
    s->opt = o;
    s->stream = cuda_stream;
    *out = s;
    return STEPS_OK;
}

void steps_server_destroy(steps_server *srv) { delete srv; }

int steps_server_submit(steps_server *srv, const steps_sim *proto, uint64_t seed, const int32_t *counts,
                        double t_end, int64_t *job) {
    if (!srv || !proto || !counts || !job) {
        steps::set_error("steps_server_submit: NULL argument");
        return STEPS_ERR_ARG;
    }
    if (!std::isfinite(t_end) || t_end < 0.0) {
        steps::set_error("steps_server_submit: t_end must be finite and >= 0");
        return STEPS_ERR_ARG;
    }
    int64_t nt = 0;
    int32_t ns = 0;
    int rc = steps_sim_shape(proto, &nt, &ns);
    if (rc) return rc;
    int grp = 0;
    rc = group_of(srv, proto, &grp);
    if (rc) return rc;
    Job j;
    j.proto = proto;
    j.seed = seed;
    j.t_end = t_end;
    try {
        // everything that can fail first; then the job is stored without reallocation
        j.counts.assign(counts, counts + (size_t)ns * (size_t)nt);
        srv->jobs.reserve(srv->jobs.size() + 1);
        srv->job_group.reserve(srv->job_group.size() + 1);
        srv->queue.push_back((int64_t)srv->jobs.size());
    } catch (const std::bad_alloc &) {
        steps::set_error("steps_server_submit: out of host memory");
        return STEPS_ERR_OOM;
    }
    srv->jobs.push_back(std::move(j));
    srv->job_group.push_back(grp);
    *job = (int64_t)srv->jobs.size() - 1;
    return STEPS_OK;
}

int steps_server_step(steps_server *srv, int32_t *running, int32_t *finished) {
    if (!srv) {
        steps::set_error("steps_server_step: NULL argument");
        return STEPS_ERR_ARG;
    }
    int32_t nfin = 0;
    // admission: first come first served, by slots and device-memory budget
    while (!srv->queue.empty() && srv->n_running < srv->opt.max_jobs) {
        const int64_t id = srv->queue.front();
        int64_t need = 0;
        int rc = steps_sim_device_bytes(srv->jobs[(size_t)id].proto, &need);
        if (rc) return rc;
        if (srv->n_running > 0 && srv->opt.device_budget > 0 && srv->bytes_running + need > srv->opt.device_budget)
            break;
        rc = admit(srv, id);
        if (rc) return rc;
        srv->queue.pop_front();
    }
    // jobs at their t_end (nothing to run, or finished last round) leave
    auto sweep = [&](Group &g) -> int {
        std::vector<int64_t> keep;
        for (int64_t id : g.running) {
            Job &j = srv->jobs[(size_t)id];
            double t = 0.0;
            steps_get_time(j.sim, &t);
            steps_get_windows(j.sim, &j.windows, nullptr);
            j.t = t;
            if (!(t < j.t_end - 1e-12 * std::max(j.t_end, 1e-30))) {
                int rc = retire(srv, id);
                if (rc) return rc;
                ++nfin;
                g.valid = false;
            } else {
                keep.push_back(id);
            }
        }
        g.running.swap(keep);
        if (!g.valid) srv->drop_batch(g);
        return STEPS_OK;
    };
    for (Group &g : srv->groups) {
        int rc = sweep(g);
        if (rc) return rc;
    }
    // one round: every group's batch moves its jobs by up to wave_windows
    // windows on their own grids; the groups' streams run at the same time
    bool any = false;
    int rc_first = STEPS_OK;
    for (Group &g : srv->groups) {
        g.enqueued = false;
        if (g.running.empty()) continue;
        if (!g.valid) {
            srv->drop_batch(g);
            std::vector<steps_sim *> members;
            for (int64_t id : g.running) members.push_back(srv->jobs[(size_t)id].sim);
            steps_batch_options bo;
            steps_batch_options_default(&bo);
            bo.block = srv->opt.block;
            bo.specialize = srv->opt.specialize;
            int rc = steps_batch_create(members.data(), (int32_t)members.size(), &bo, g.stream, &g.batch);
            if (rc) {
                rc_first = rc;
                break;
            }
            g.valid = true;
            ++srv->rebuilds;
        }
        std::vector<double> target;
        for (int64_t id : g.running) {
            Job &j = srv->jobs[(size_t)id];
            double t = 0.0, tau = 0.0;
            steps_get_time(j.sim, &t);
            steps_get_tau(j.sim, &tau);
            const double tg = std::isfinite(tau) ? t + (double)srv->opt.wave_windows * tau : j.t_end;
            target.push_back(std::min(j.t_end, tg));
        }
        int rc = steps::batch_enqueue(g.batch, target.data());
        if (rc) {
            rc_first = rc;
            break;
        }
        g.enqueued = true;
        any = true;
    }
    // wait for every enqueued batch, even after an error
    for (Group &g : srv->groups) {
        if (!g.enqueued) continue;
        int rc = steps::batch_finish(g.batch);
        if (rc && rc_first == STEPS_OK) rc_first = rc;
        g.enqueued = false;
    }
    if (rc_first) return rc_first;
    if (any) ++srv->rounds;
    for (Group &g : srv->groups) {
        int rc = sweep(g);
        if (rc) return rc;
    }
    if (running) *running = srv->n_running;
    if (finished) *finished = nfin;
    return STEPS_OK;
}

int steps_server_job_state(const steps_server *srv, int64_t job, int32_t *state, uint64_t *windows, double *t) {
    if (!srv || !valid_job(srv, job)) {
        steps::set_error("steps_server_job_state: unknown job");
        return STEPS_ERR_ARG;
    }
    const Job &j = srv->jobs[(size_t)job];
    if (state) *state = j.state;
    if (windows) *windows = j.windows;
    if (t) *t = j.t;
    return STEPS_OK;
}

int steps_server_take_result(steps_server *srv, int64_t job, int32_t *counts_out) {
    if (!srv || !valid_job(srv, job)) {
        steps::set_error("steps_server_take_result: unknown job");
        return STEPS_ERR_ARG;
    }
    Job &j = srv->jobs[(size_t)job];
    if (j.state != 2) {
        steps::set_error(j.state == 3 ? "steps_server_take_result: result already taken"
                                      : "steps_server_take_result: job not finished");
        return STEPS_ERR_STATE;
    }
    if (counts_out) std::memcpy(counts_out, j.counts.data(), j.counts.size() * sizeof(int32_t));
    j.counts.clear();
    j.counts.shrink_to_fit();
    j.state = 3;
    return STEPS_OK;
}

int steps_server_stats(const steps_server *srv, uint64_t *rounds, uint64_t *rebuilds, uint64_t *launches,
                       int32_t *queued, int32_t *running, int64_t *device_bytes) {
    if (!srv) {
        steps::set_error("steps_server_stats: NULL argument");
        return STEPS_ERR_ARG;
    }
    if (rounds) *rounds = srv->rounds;
    if (rebuilds) *rebuilds = srv->rebuilds;
    if (launches) {
        uint64_t l = srv->launches;
        for (const Group &g : srv->groups) {
            uint64_t bl = 0;
            if (g.batch && steps_batch_info(g.batch, nullptr, &bl, nullptr) == STEPS_OK) l += bl;
        }
        *launches = l;
    }
    if (queued) *queued = (int32_t)srv->queue.size();
    if (running) *running = srv->n_running;
    if (device_bytes) *device_bytes = srv->bytes_running;
    return STEPS_OK;
}

}  // extern "C"
