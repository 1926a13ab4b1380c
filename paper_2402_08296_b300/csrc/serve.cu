// Serving: a request loop that solves Poisson problems as they arrive.
//
// ddg_submit queues a request (mesh, data coefficients, solver options) and
// returns a ticket; a scheduler thread owned by the context admits queued
// requests while the estimate of their device memory fits the context's HBM
// budget (and fewer than max_active are in flight), sets each admitted request
// up on a CUDA stream of its own (upload, assembly, decomposition,
// preconditioner), and then advances every in-flight flexible-CG solve a batch
// of iterations at a time without blocking: kernels of different requests run
// concurrently on the GPU, and a request that arrives while others are running
// starts as soon as a slot and memory are free (continuous batching).  Krylov
// state stays on the device between batches.  ddg_poll returns DDG_PENDING
// until the request has finished, then its report and solution.
//
// With fused GNN launches, DDM-GNN requests that share a model run in groups: every step advances
// each member by one FCG iteration, and the local GNN solves of all members run
// as one fused launch per message-passing block over the subdomains of every
// member (schedule 3, chunk width GROUP_T), between the members' restriction
// and gluing kernels on their own streams.  Members join and leave the group
// between steps.  Results are bitwise the same as a stand-alone ddg_fcg_solve
// with the same GNN schedule, since every CTA only touches one request's
// buffers and every sum runs in a fixed order.  This mode is chosen with
// ddg_serve_config; by default every request runs on its own stream with its
// FCG periods replayed as CUDA graphs, which measured faster on one B300.
#include "ddg_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <cstdlib>
#include <thread>

namespace ddg {

static constexpr int MAX_GROUP_REQUESTS = 32;  // problems of one fused GNN launch

static double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct ServeRequest {
    uint64_t ticket = 0;
    std::vector<double> xy;
    std::vector<int32_t> tri;
    double r9[9];
    ddg_solve_opts opts;
    size_t est_bytes = 0;
    ddg_problem *p = nullptr;
    FcgRun *run = nullptr;
    int32_t status = DDG_PENDING;
    bool grouped = false;       // member of the fused GNN group
    bool marked = false;        // a flag copy is queued (fcg_check can observe it)
    cudaEvent_t ev_pre = nullptr;
    ddg_solve_report rep{};
    std::vector<double> x;
    std::string err;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
};

struct Server {
    ddg_ctx *ctx = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ServeRequest *> pending;
    std::vector<ServeRequest *> active;
    std::map<uint64_t, ServeRequest *> finished;
    std::set<uint64_t> live;  // tickets submitted and not yet collected
    bool stop = false;
    uint64_t next_ticket = 1;
    int max_active = 64;
    int max_pending = 65536;
    size_t reserved = 0;
    std::vector<double> latencies;
    uint64_t completed = 0, failed = 0;
    double t_first_submit = -1.0, t_last_done = 0.0;
    // fused GNN groups (used by the scheduler thread only): two, stepped alternately, so that
    // one group's GNN launches overlap the other group's Krylov kernels
    std::atomic<bool> fuse{false};  // DDM-GNN requests join fused groups (ddg_serve_config)
    bool fuse_ready = false;  // the groups' streams, events and descriptor buffers exist
    struct Group {
        std::vector<ServeRequest *> members;
        std::vector<ddg_problem *> uploaded;  // members of the last descriptor upload
        cudaStream_t stream = nullptr;
        cudaEvent_t ev_gnn = nullptr;
        static constexpr int DEPTH = 4;       // steps queued ahead of the host
        cudaEvent_t ev_step[DEPTH] = {};
        int steps = 0, steps_done = 0;
        ChunkArgs *args = nullptr;            // device descriptors of the members
    };
    static constexpr int NGROUPS = 2;
    Group groups[NGROUPS];
    Allocs gallocs;
    size_t grouped() const {
        size_t n = 0;
        for (const Group &g : groups) n += g.members.size();
        return n;
    }
};

static constexpr int GROUP_POLL = 4;  // group steps between flag copies of a member

// device memory of one request: mesh, matrix, decomposition, Krylov rings, and the
// preconditioner (band factors for DDM-LU, latents for DDM-GNN) plus the coarse matrix
static size_t estimate_bytes(int n_nodes, const ddg_solve_opts &o) {
    const size_t per_node = o.kind == DDG_DDM_LU ? 3200 : 1600;
    const long long K = o.K > 0 ? o.K : std::max(1, n_nodes / 1000);
    return (size_t)n_nodes * per_node + (size_t)K * K * 16 + (4u << 20);
}

static void finish(Server *S, ServeRequest *q, int32_t status, const std::string &err) {
    q->status = status;
    q->err = err;
    q->t_done = now_ms();
    if (q->grouped) {
        // every queued step that holds this member has ended once its stream and its group's
        // stream are idle; then the member leaves the group
        for (Server::Group &g : S->groups) {
            if (std::find(g.members.begin(), g.members.end(), q) == g.members.end()) continue;
            if (q->p) cudaStreamSynchronize(q->p->stream);
            if (g.stream) cudaStreamSynchronize(g.stream);
            g.uploaded.clear();
            g.members.erase(std::remove(g.members.begin(), g.members.end(), q), g.members.end());
        }
        q->grouped = false;
    }
    if (q->ev_pre) {
        cudaEventDestroy(q->ev_pre);
        q->ev_pre = nullptr;
    }
    if (q->run) {
        fcg_delete(q->run);
        q->run = nullptr;
    }
    if (q->p) {
        ddg_problem_destroy(q->p);
        q->p = nullptr;
    }
    q->xy.clear();
    q->xy.shrink_to_fit();
    q->tri.clear();
    q->tri.shrink_to_fit();
    std::lock_guard<std::mutex> lock(S->mu);
    S->reserved -= q->est_bytes;
    S->active.erase(std::remove(S->active.begin(), S->active.end(), q), S->active.end());
    S->finished[q->ticket] = q;
    if (status == DDG_OK || status == DDG_NOT_CONVERGED || status == DDG_BREAKDOWN) {
        S->latencies.push_back(q->t_done - q->t_submit);
        ++S->completed;
        S->t_last_done = q->t_done;
    } else {
        ++S->failed;
    }
    S->cv.notify_all();
}

static int32_t start(Server *S, ServeRequest *q) {
    ddg_ctx *c = S->ctx;
    const int n = (int)(q->xy.size() / 2), t = (int)(q->tri.size() / 3);
    cudaStream_t st = nullptr;
    DDG_CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    int32_t s = problem_create(c, n, q->xy.data(), t, q->tri.data(), nullptr, st, true, &q->p);
    if (s != DDG_OK) {
        cudaStreamDestroy(st);
        return s;
    }
    DDG_TRY(ddg_assemble_poly(q->p, q->r9));
    int K = q->opts.K > 0 ? q->opts.K : std::max(1, (int)std::lround(q->p->nf / 1000.0));
    K = std::min(K, q->p->nf);
    DDG_TRY(ddg_partition(q->p, K, q->opts.overlap, nullptr));
    DDG_TRY(ddg_setup_precond(q->p, q->opts.kind, q->opts.model, q->opts.flags));
    q->x.resize(n);
    // the smaller group (fewer graph nodes) takes the request, if compatible
    Server::Group *join = nullptr;
    if (S->fuse && q->opts.kind == DDG_DDM_GNN && q->opts.model->d == DSS_D) {
        DDG_TRY(dss_group_prepare(q->p));
        long long best = -1;
        for (Server::Group &g : S->groups) {
            if ((int)g.members.size() >= MAX_GROUP_REQUESTS) continue;
            if (!g.members.empty() && !dss_group_compatible(g.members[0]->p, q->p)) continue;
            long long load = 0;
            for (ServeRequest *m : g.members) load += m->p->sum_loc;
            if (best < 0 || load < best) {
                best = load;
                join = &g;
            }
        }
    }
    q->run = fcg_new();
    DDG_TRY(fcg_begin(q->run, q->p, nullptr, q->opts.rtol, q->opts.max_iter, q->opts.m_trunc));
    if (join) {
        DDG_CU(cudaEventCreateWithFlags(&q->ev_pre, cudaEventDisableTiming));
        q->grouped = true;
        join->members.push_back(q);
        return DDG_OK;
    }
    return fcg_launch_batch(q->run);
}

// one fused step of group G: every member that still has iterations to run advances by one
static int32_t group_step(Server::Group &G, bool *launched) {
    std::vector<ServeRequest *> mem;
    for (ServeRequest *q : G.members)
        if (fcg_iterations_launched(q->run) < fcg_max_iter(q->run)) mem.push_back(q);
    *launched = false;
    if (mem.empty()) return DDG_OK;
    std::vector<ddg_problem *> ps;
    std::vector<const double *> rs;
    std::vector<const int *> stops;
    for (ServeRequest *q : mem) {
        DDG_TRY(fcg_group_pre(q->run));
        DDG_CU(cudaEventRecord(q->ev_pre, q->p->stream));
        DDG_CU(cudaStreamWaitEvent(G.stream, q->ev_pre, 0));
        ps.push_back(q->p);
        rs.push_back(fcg_residual(q->run));
        stops.push_back(fcg_flag(q->run));
    }
    const bool upload = ps != G.uploaded;
    DDG_TRY(dss_group_launch(ps.data(), rs.data(), stops.data(), (int)ps.size(), G.args, upload, G.stream));
    G.uploaded = ps;
    DDG_CU(cudaEventRecord(G.ev_gnn, G.stream));
    for (ServeRequest *q : mem) {
        DDG_CU(cudaStreamWaitEvent(q->p->stream, G.ev_gnn, 0));
        DDG_TRY(fcg_group_post(q->run));
        if (!q->marked && (fcg_group_since_mark(q->run) >= GROUP_POLL ||
                           fcg_iterations_launched(q->run) >= fcg_max_iter(q->run))) {
            DDG_TRY(fcg_group_mark(q->run));
            q->marked = true;
        }
    }
    DDG_CU(cudaEventRecord(G.ev_step[G.steps % Server::Group::DEPTH], G.stream));
    ++G.steps;
    *launched = true;
    return DDG_OK;
}

// one pass of the scheduler; false once it has been asked to stop and nothing is left
static bool loop_once(Server *S) {
    std::vector<ServeRequest *> admit;
    std::vector<ServeRequest *> act;
    {
        std::unique_lock<std::mutex> lock(S->mu);
        if (S->stop && S->pending.empty() && S->active.empty()) return false;
        while (!S->pending.empty() && (int)S->active.size() + (int)admit.size() < S->max_active) {
            ServeRequest *q = S->pending.front();
            const size_t budget = S->ctx->budget;
            const bool nothing_running = S->active.empty() && admit.empty();
            // wait for memory unless nothing runs (then the request proceeds and may fail with DDG_OOM)
            if (budget && S->reserved + q->est_bytes > budget && !nothing_running) break;
            S->pending.pop_front();
            S->reserved += q->est_bytes;
            q->t_admit = now_ms();
            admit.push_back(q);
            S->active.push_back(q);
        }
        act = S->active;
    }
    bool progressed = !admit.empty();
    for (ServeRequest *q : admit) {
        int32_t s = api_guard([&]() -> int32_t { return start(S, q); });
        if (s != DDG_OK) finish(S, q, s, last_error_cstr());
    }
    for (ServeRequest *q : act) {  // requests on their own (group members are handled below)
        // (admitted this round: started above, possibly already finished and collected)
        if (std::find(admit.begin(), admit.end(), q) != admit.end() || !q->run || q->grouped) continue;
        bool ready = false, done = false;
        int32_t s = fcg_check(q->run, false, &ready, &done);
        if (s != DDG_OK) {
            finish(S, q, s, last_error_cstr());
            progressed = true;
            continue;
        }
        if (!ready) continue;
        progressed = true;
        if (done) {
            int32_t fs = fcg_end(q->run, q->x.data(), &q->rep);
            q->rep.solve_ms = now_ms() - q->t_admit;  // wall time from admission to the result
            finish(S, q, fs, fs == DDG_OK ? "" : last_error_cstr());
        } else {
            s = fcg_launch_batch(q->run);
            if (s != DDG_OK) finish(S, q, s, last_error_cstr());
        }
    }
    // fused GNN groups: alternately queue one step of each while fewer than DEPTH are in flight
    for (bool any = true; any;) {
        any = false;
        for (Server::Group &G : S->groups) {
            if (G.members.empty()) continue;
            while (G.steps_done < G.steps &&
                   cudaEventQuery(G.ev_step[G.steps_done % Server::Group::DEPTH]) == cudaSuccess)
                ++G.steps_done;
            cudaGetLastError();
            if (G.steps - G.steps_done >= Server::Group::DEPTH) continue;
            bool launched = false;
            int32_t s = api_guard([&]() -> int32_t { return group_step(G, &launched); });
            if (s != DDG_OK) {  // a launch failed: fail every member
                std::vector<ServeRequest *> g = G.members;
                for (ServeRequest *q : g) finish(S, q, s, last_error_cstr());
                progressed = true;
                continue;
            }
            if (launched) any = progressed = true;
        }
    }
    for (Server::Group &G : S->groups) {
        for (ServeRequest *q : std::vector<ServeRequest *>(G.members)) {
            if (!q->marked) continue;
            bool ready = false, done = false;
            int32_t s = fcg_check(q->run, false, &ready, &done);
            if (s != DDG_OK) {
                finish(S, q, s, last_error_cstr());
                progressed = true;
                continue;
            }
            if (!ready) continue;
            q->marked = false;
            progressed = true;
            if (done) {
                int32_t fs = fcg_end(q->run, q->x.data(), &q->rep);
                q->rep.solve_ms = now_ms() - q->t_admit;
                finish(S, q, fs, fs == DDG_OK ? "" : last_error_cstr());
            }
        }
    }
    if (!progressed) {
        std::unique_lock<std::mutex> lock(S->mu);
        S->cv.wait_for(lock, std::chrono::microseconds(S->active.empty() ? 2000 : 30));
    }
    return true;
}

// The scheduler thread.  Calls that allocate host memory for a request are guarded above and
// fail that request with a status; anything else that throws (host memory exhausted in the
// scheduler's own bookkeeping) ends only the pass, and the next pass retries.
static void loop(Server *S) {
    cudaSetDevice(S->ctx->device);
    for (;;) {
        try {
            if (!loop_once(S)) break;
        } catch (...) {
            std::this_thread::sleep_for(std::chrono::milliseconds(1));
        }
    }
}

void server_stop(ddg_ctx *c) {
    Server *S = c->server;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    for (auto &kv : S->finished) delete kv.second;
    for (Server::Group &g : S->groups) {
        if (g.stream) cudaStreamSynchronize(g.stream);
        for (int k = 0; k < Server::Group::DEPTH; ++k)
            if (g.ev_step[k]) cudaEventDestroy(g.ev_step[k]);
        if (g.ev_gnn) cudaEventDestroy(g.ev_gnn);
        if (g.stream) cudaStreamDestroy(g.stream);
    }
    dfree_all(c, S->gallocs);
    delete S;
    c->server = nullptr;
}

static Server *server_get(ddg_ctx *c) {
    std::lock_guard<std::mutex> lock(c->server_mu);
    if (!c->server) {
        Server *S = new Server();
        S->ctx = c;
        cudaSetDevice(c->device);
        bool ok = true;
        for (Server::Group &g : S->groups) {
            ok = ok && cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&g.ev_gnn, cudaEventDisableTiming) == cudaSuccess;
            for (int k = 0; k < Server::Group::DEPTH && ok; ++k)
                ok = cudaEventCreateWithFlags(&g.ev_step[k], cudaEventDisableTiming) == cudaSuccess;
            ok = ok && dalloc(c, S->gallocs, reinterpret_cast<char **>(&g.args), dss_group_args_bytes()) == DDG_OK;
        }
        S->fuse_ready = ok;  // without them every request runs on its own (still on the GPU)
        c->server = S;
        S->th = std::thread(loop, S);
    }
    return c->server;
}

}  // namespace ddg

using namespace ddg;

extern "C" {

int32_t ddg_serve_config(ddg_ctx *c, int32_t max_active, int32_t fuse_gnn, int32_t max_pending) {
    return api_guard([&]() -> int32_t {
        clear_error();
        if (!c || max_active < 1 || (fuse_gnn != 0 && fuse_gnn != 1) || max_pending < 1) {
            set_error("ddg_serve_config: bad arguments");
            return DDG_INVALID_ARG;
        }
        Server *S = server_get(c);
        std::lock_guard<std::mutex> lock(S->mu);
        S->max_active = max_active;
        S->max_pending = max_pending;
        // the scheduler reads `fuse` when it starts a request: switching only affects later ones
        S->fuse = fuse_gnn != 0 && S->fuse_ready;
        return DDG_OK;
    });
}

int32_t ddg_submit(ddg_ctx *c, int32_t n_nodes, const double *xy, int32_t n_tri, const int32_t *tri,
                   const double r[9], const ddg_solve_opts *opts, uint64_t *ticket) {
    return api_guard([&]() -> int32_t {
        clear_error();
        if (!c || !xy || !tri || !r || !opts || !ticket || n_nodes < 3 || n_tri < 1) {
            set_error("ddg_submit: bad arguments");
            return DDG_INVALID_ARG;
        }
        if ((opts->kind == DDG_DDM_GNN && !opts->model) || opts->rtol <= 0.0 || opts->max_iter < 1 ||
            opts->m_trunc < 1 || opts->overlap < 0) {
            set_error("ddg_submit: bad solver options");
            return DDG_INVALID_ARG;
        }
        ServeRequest *q = new ServeRequest();
        q->xy.assign(xy, xy + 2 * (size_t)n_nodes);
        q->tri.assign(tri, tri + 3 * (size_t)n_tri);
        std::memcpy(q->r9, r, sizeof(q->r9));
        q->opts = *opts;
        q->est_bytes = estimate_bytes(n_nodes, *opts);
        q->t_submit = now_ms();
        Server *S = server_get(c);
        std::lock_guard<std::mutex> lock(S->mu);
        if ((int)S->pending.size() >= S->max_pending) {
            delete q;
            set_error("ddg_submit: the admission queue is full");
            return DDG_BUSY;
        }
        q->ticket = S->next_ticket++;
        S->live.insert(q->ticket);
        if (S->t_first_submit < 0.0) S->t_first_submit = q->t_submit;
        S->pending.push_back(q);
        *ticket = q->ticket;
        S->cv.notify_all();
        return DDG_OK;
    });
}

int32_t ddg_poll(ddg_ctx *c, uint64_t ticket, ddg_solve_report *report, double *x_host) {
    return api_guard([&]() -> int32_t {
        clear_error();
        if (!c) {
            set_error("ddg_poll: NULL context");
            return DDG_INVALID_ARG;
        }
        Server *S = server_get(c);
        ServeRequest *q = nullptr;
        {
            std::lock_guard<std::mutex> lock(S->mu);
            auto it = S->finished.find(ticket);
            if (it == S->finished.end()) {
                if (!S->live.count(ticket)) {
                    set_error("ddg_poll: unknown or already collected ticket");
                    return DDG_INVALID_ARG;
                }
                return DDG_PENDING;
            }
            q = it->second;
            S->finished.erase(it);
            S->live.erase(ticket);
        }
        if (report) *report = q->rep;
        if (x_host && !q->x.empty()) std::memcpy(x_host, q->x.data(), sizeof(double) * q->x.size());
        int32_t st = q->status;
        if (!q->err.empty()) set_error(q->err);
        delete q;
        return st;
    });
}

int32_t ddg_serve_stats(ddg_ctx *c, ddg_serve_summary *out) {
    return api_guard([&]() -> int32_t {
        clear_error();
        if (!c || !out) {
            set_error("ddg_serve_stats: bad arguments");
            return DDG_INVALID_ARG;
        }
        Server *S = server_get(c);
        std::lock_guard<std::mutex> lock(S->mu);
        std::memset(out, 0, sizeof(*out));
        out->completed = S->completed;
        out->failed = S->failed;
        out->pending = S->pending.size();
        out->active = S->active.size();
        out->reserved_bytes = S->reserved;
        out->device_bytes = c->in_use;
        if (!S->latencies.empty()) {
            std::vector<double> l = S->latencies;
            std::sort(l.begin(), l.end());
            auto pct = [&](double f) { return l[std::min(l.size() - 1, (size_t)(f * (l.size() - 1) + 0.5))]; };
            out->p50_ms = pct(0.50);
            out->p99_ms = pct(0.99);
            double span = S->t_last_done - S->t_first_submit;
            out->solves_per_s = span > 0.0 ? S->completed / (span / 1e3) : 0.0;
        }
        return DDG_OK;
    });
}

}  // extern "C"
