// Serving runtime: continuous batching of radiative-transfer solve requests.
//
// Requests of any grid size, direction count, eps and g are queued as they
// arrive.  A scheduler admits the oldest waiting request as soon as a worker
// slot is free and its estimated device footprint fits in the budget (admission
// by HBM footprint); each slot runs on its own CUDA stream with stream-ordered
// allocation, so the solves of all admitted requests overlap on the GPU and
// one request's set-up or release never synchronises the others.  A finished
// request releases its slot and its bytes at once and the next one is admitted
// -- continuous batching rather than batch-synchronous rounds.  Results are
// computed with the same deterministic kernels as a lone solve, so each result
// is bit-identical alone and in the mix.  Faults stay per request: a malformed
// medium, an injected allocation failure or a cancellation ends that request
// with its status; the others continue.
//
// Grouped mode: the admitted requests form one lockstep group on one stream.
// Setup threads build each admitted request's context and vectors and hand it
// to the group thread, which adds it to the group at the next round; every
// round advances all running solves by one Arnoldi step in shared launches
// (the rounds of rte_solve_group), and a solve that finishes is reconstructed,
// copied out and released at once.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include <cmath>

#include "rte_internal.h"

namespace rte {
namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    int64_t id = 0;
    int I = 0, M = 0;
    std::vector<double> sT, sa, q, eps, inflow;
    int eps_is_scalar = 1;
    double g = 0.0;
    rte_solve_opts opts{};
    int use_net = 0;
    int net = -1;                     // index of the server's network for (I, M), -1: block Jacobi
    size_t footprint = 0;
    Clock::time_point t_submit, t_start, t_end;
    volatile int cancel = 0;
    bool done = false;
    rte_status status = RTE_OK;
    rte_solve_info info{};
    std::vector<double> psi;          // [M][N]
    std::string err;
    // grouped mode: the request's context and vectors while it runs
    rte_ctx* ctx = nullptr;
    double* x = nullptr;
    double* psi_dev = nullptr;
};

}  // namespace
}  // namespace rte

struct rte_server {
    rte_server_config cfg{};
    int device = 0;
    std::vector<mgnet_config> net_cfg;         // the networks the server holds, one per M
    std::vector<std::vector<mgnet*>> nets;     // [slot][network]: a copy per slot (one stream each)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<rte::Job>> queue;
    std::map<int64_t, std::shared_ptr<rte::Job>> jobs;
    size_t bytes_in_use = 0;
    int active = 0;
    int64_t next_id = 1;
    bool stopping = false;
    std::vector<std::thread> workers;
    int64_t completed = 0;
    // grouped mode
    cudaStream_t gst = nullptr;
    std::vector<mgnet*> gnets;                 // grouped mode: one copy per network on gst
    std::deque<std::shared_ptr<rte::Job>> setup_q;   // admitted, waiting for a setup thread
    std::vector<std::shared_ptr<rte::Job>> ready;    // set up, waiting to join the group
    std::condition_variable cv_setup, cv_group;
};

namespace rte {
namespace {

// Device bytes a solve holds: D (FP64) and R (FP32) blocks, per-cell tables,
// the eigenbases of its materials (FP64 and FP32, plain and transposed), b and
// the operator scratch, the Krylov basis (FP64) and MgNet outputs (FP32).
size_t footprint(int I, int M, int restart, bool net, size_t nmat) {
    const size_t N = (size_t)I * I, n2 = 2 * (size_t)M, n = n2 * N;
    size_t b = N * n2 * n2 * (8 + 4);
    b += n * 8 * 6;                                    // b, trace scratch (2n), w, tmp, x
    b += (size_t)(restart + 1) * n * 8 + (size_t)restart * n * 4;
    b += N * 64 + nmat * (size_t)M * n2 * (8 + 8 + 4 + 4) + nmat * n2 * 8;   // per-cell and basis tables
    if (net) b += n * 4 * 16;                          // network activations (upper bound)
    return b + (64u << 20);
}

// materials of a request: distinct 1 - gamma = eps^2 sigma_a / sigma_T, as rte_setup counts them
size_t count_materials(const Job& j) {
    std::vector<double> w;
    w.reserve(j.sT.size());
    for (size_t c = 0; c < j.sT.size(); ++c) {
        const double e = j.eps_is_scalar ? j.eps[0] : j.eps[c];
        const double v = e * e * j.sa[c] / j.sT[c];
        if (std::isfinite(v)) w.push_back(v);   // a malformed medium fails at set-up
    }
    std::sort(w.begin(), w.end());
    return (size_t)(std::unique(w.begin(), w.end()) - w.begin());
}

bool valid_request(const rte_request* r, std::string& why) {
    if (!r->sigma_T || !r->sigma_a || !r->q || !r->eps) { why = "NULL medium array"; return false; }
    if (r->I < 1 || r->I > 8192 || r->M < 4 || r->M % 4 || r->M > 80) { why = "bad I or M"; return false; }
    if (!(std::fabs(r->g) < 1.0)) { why = "need |g| < 1"; return false; }
    return true;
}

// The network for a request of I x I cells and M directions: the one with
// the same M whose V-cycle depth divides I; -1 when there is none.
int pick_net(const rte_server* s, int I, int M) {
    for (size_t k = 0; k < s->net_cfg.size(); ++k) {
        const mgnet_config& c = s->net_cfg[k];
        if (c.M == M && I % (1 << (c.levels - 1)) == 0) return (int)k;
    }
    return -1;
}

void worker_main(rte_server* s, int slot) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    while (true) {
        std::shared_ptr<Job> job;
        bool admitted = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                if (s->stopping) return true;
                if (s->queue.empty()) return false;
                const auto& head = s->queue.front();
                return head->cancel || s->bytes_in_use + head->footprint <= s->cfg.max_device_bytes;
            });
            if (s->stopping && s->queue.empty()) break;
            if (s->stopping) break;
            job = s->queue.front();
            s->queue.pop_front();
            admitted = !job->cancel;
            if (admitted) {
                s->bytes_in_use += job->footprint;
                ++s->active;
            }
        }
        job->t_start = Clock::now();
        if (!admitted) {
            job->status = RTE_ECANCELLED;
            job->err = "cancelled before admission";
        } else if (s->cfg.inject_alloc_failure_id == job->id) {
            job->status = RTE_ENOMEM;          // host-side fault injection for tests
            job->err = "injected allocation failure";
        } else {
            rte_ctx* ctx = nullptr;
            rte_grid grid{job->I};
            rte_quadrature quad{job->M};
            job->status = rte_setup(&grid, &quad, job->sT.data(), job->sa.data(), job->q.data(),
                                    job->eps.data(), job->eps_is_scalar, job->g,
                                    job->inflow.empty() ? nullptr : job->inflow.data(), st, &ctx);
            if (job->status == RTE_OK) {
                const int64_t n = (int64_t)2 * job->M * job->I * job->I;
                double* x = nullptr;
                double* psi = nullptr;
                cudaError_t e = pool_malloc(reinterpret_cast<void**>(&x), n * sizeof(double), st);
                if (e == cudaSuccess) e = pool_malloc(reinterpret_cast<void**>(&psi), (size_t)job->M * job->I * job->I * sizeof(double), st);
                if (e != cudaSuccess) {
                    job->status = RTE_ENOMEM;
                    job->err = cudaGetErrorString(e);
                } else {
                    job->opts.cancel = &job->cancel;
                    mgnet* pc = job->net >= 0 ? s->nets[slot][job->net] : nullptr;
                    job->status = rte_solve(ctx, pc, &job->opts, x, &job->info);
                    if (job->status == RTE_OK || job->status == RTE_ENOTCONV) {
                        rte_reconstruct(ctx, x, psi);
                        job->psi.resize((size_t)job->M * job->I * job->I);
                        cudaMemcpyAsync(job->psi.data(), psi, job->psi.size() * sizeof(double),
                                        cudaMemcpyDeviceToHost, st);
                        cudaStreamSynchronize(st);
                    }
                    if (job->status != RTE_OK) job->err = rte_last_error(ctx);
                }
                if (x) cudaFreeAsync(x, st);
                if (psi) cudaFreeAsync(psi, st);
                rte_destroy(ctx);
            } else {
                job->err = rte_last_error(nullptr);
            }
        }
        job->t_end = Clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (admitted) {
                s->bytes_in_use -= job->footprint;
                --s->active;
            }
            job->done = true;
            ++s->completed;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    cudaStreamDestroy(st);
}

// Releases a finished request (grouped mode): bytes, slot, completion.
void finish_job(rte_server* s, const std::shared_ptr<Job>& job, bool admitted) {
    job->t_end = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (admitted) {
            s->bytes_in_use -= job->footprint;
            --s->active;
        }
        job->done = true;
        ++s->completed;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

// Grouped mode, admission: the oldest waiting request goes to the setup
// threads when the group has a free slot and its footprint fits.
void admit_main(rte_server* s) {
    while (true) {
        std::shared_ptr<Job> job;
        bool admitted = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                if (s->stopping) return true;
                if (s->queue.empty()) return false;
                const auto& head = s->queue.front();
                return head->cancel || (s->active < s->cfg.slots &&
                                        s->bytes_in_use + head->footprint <= s->cfg.max_device_bytes);
            });
            if (s->stopping) break;
            job = s->queue.front();
            s->queue.pop_front();
            admitted = !job->cancel;
            if (admitted) {
                s->bytes_in_use += job->footprint;
                ++s->active;
            }
            job->t_start = Clock::now();
            if (admitted) {
                s->setup_q.push_back(job);
                s->cv_setup.notify_one();
                continue;
            }
        }
        job->status = RTE_ECANCELLED;
        job->err = "cancelled before admission";
        finish_job(s, job, false);
    }
}

// Grouped mode, set-up: context, solution and output vectors on the group's
// stream, then hand-over to the group thread.
void setup_main(rte_server* s) {
    cudaSetDevice(s->device);
    while (true) {
        std::shared_ptr<Job> job;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_setup.wait(lk, [&] { return s->stopping || !s->setup_q.empty(); });
            if (s->stopping) break;
            job = s->setup_q.front();
            s->setup_q.pop_front();
        }
        bool ok = false;
        if (s->cfg.inject_alloc_failure_id == job->id) {
            job->status = RTE_ENOMEM;          // host-side fault injection for tests
            job->err = "injected allocation failure";
        } else {
            rte_grid grid{job->I};
            rte_quadrature quad{job->M};
            job->status = rte_setup(&grid, &quad, job->sT.data(), job->sa.data(), job->q.data(), job->eps.data(),
                                    job->eps_is_scalar, job->g, job->inflow.empty() ? nullptr : job->inflow.data(),
                                    s->gst, &job->ctx);
            if (job->status == RTE_OK) {
                const int64_t n = (int64_t)2 * job->M * job->I * job->I;
                cudaError_t e = pool_malloc(reinterpret_cast<void**>(&job->x), n * sizeof(double), s->gst);
                if (e == cudaSuccess)
                    e = pool_malloc(reinterpret_cast<void**>(&job->psi_dev), (size_t)job->M * job->I * job->I * sizeof(double), s->gst);
                if (e != cudaSuccess) {
                    job->status = RTE_ENOMEM;
                    job->err = cudaGetErrorString(e);
                } else {
                    ok = true;
                }
            } else {
                job->err = rte_last_error(nullptr);
            }
        }
        if (ok) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->ready.push_back(job);
            s->cv_group.notify_one();
        } else {
            if (job->psi_dev) cudaFreeAsync(job->psi_dev, s->gst);
            if (job->x) cudaFreeAsync(job->x, s->gst);
            if (job->ctx) rte_destroy(job->ctx);
            job->ctx = nullptr;
            finish_job(s, job, true);
        }
    }
}

// reconstruct psi, copy it out, free the request's device state
void complete_job(rte_server* s, const std::shared_ptr<Job>& job) {
    if (job->status == RTE_OK || job->status == RTE_ENOTCONV) {
        rte_reconstruct(job->ctx, job->x, job->psi_dev);
        job->psi.resize((size_t)job->M * job->I * job->I);
        cudaMemcpyAsync(job->psi.data(), job->psi_dev, job->psi.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        s->gst);
        cudaStreamSynchronize(s->gst);
    }
    if (job->status != RTE_OK && job->err.empty()) job->err = rte_last_error(job->ctx);
    cudaFreeAsync(job->x, s->gst);
    cudaFreeAsync(job->psi_dev, s->gst);
    rte_destroy(job->ctx);
    job->ctx = nullptr;
    finish_job(s, job, true);
}

// Grouped mode, the lockstep group: requests join between rounds and leave
// when they finish.
void group_main(rte_server* s) {
    cudaSetDevice(s->device);
    GroupRounds* rounds = nullptr;
    std::vector<std::pair<std::shared_ptr<Job>, GroupSolve*>> live;
    try {
        rounds = group_rounds_new(s->gst, s->cfg.slots);
        while (true) {
            std::vector<std::shared_ptr<Job>> joining;
            {
                std::unique_lock<std::mutex> lk(s->mu);
                if (live.empty())
                    s->cv_group.wait(lk, [&] { return s->stopping || !s->ready.empty(); });
                if (s->stopping) break;
                joining.swap(s->ready);
            }
            for (auto& job : joining) {
                job->opts.cancel = &job->cancel;
                mgnet* pc = job->net >= 0 ? s->gnets[job->net] : nullptr;
                try {
                    live.emplace_back(job, group_solve_new(job->ctx, pc, job->opts, job->x));
                } catch (const StatusError& e) {
                    job->status = e.code;
                    job->err = e.msg;
                    complete_job(s, job);
                } catch (const CudaError& e) {
                    job->status = cuda_status(nullptr, e.code, e.where);
                    job->err = e.where;
                    complete_job(s, job);
                }
            }
            std::vector<GroupSolve*> set;
            for (auto& p : live) set.push_back(p.second);
            group_rounds_step(rounds, set.data(), (int)set.size());
            for (size_t i = 0; i < live.size();) {
                if (group_solve_done(live[i].second)) {
                    auto job = live[i].first;
                    group_solve_result(live[i].second, &job->info, &job->status);
                    group_solve_free(live[i].second);
                    complete_job(s, job);
                    live.erase(live.begin() + i);
                } else {
                    ++i;
                }
            }
        }
    } catch (const CudaError& e) {
        const rte_status st = cuda_status(nullptr, e.code, e.where);
        for (auto& p : live) {
            p.first->status = st;
            p.first->err = e.where;
            group_solve_free(p.second);
            complete_job(s, p.first);
        }
        live.clear();
    } catch (const StatusError& e) {
        for (auto& p : live) {
            p.first->status = e.code;
            p.first->err = e.msg;
            group_solve_free(p.second);
            complete_job(s, p.first);
        }
        live.clear();
    }
    for (auto& p : live) {             // stopping: cancelled mid-solve
        p.first->status = RTE_ECANCELLED;
        p.first->err = "server stopped";
        group_solve_free(p.second);
        complete_job(s, p.first);
    }
    if (rounds) group_rounds_free(rounds);
}

}  // namespace
}  // namespace rte

using namespace rte;

extern "C" {

RTE_API void rte_server_config_default(rte_server_config* c) {
    if (!c) return;
    c->max_device_bytes = (size_t)64 << 30;
    c->slots = 4;
    c->inject_alloc_failure_id = -1;
    c->grouped = 0;
}

static void destroy_nets(rte_server* s) {
    for (auto& v : s->nets)
        for (mgnet* m : v) mgnet_destroy(m);
    s->nets.clear();
    for (mgnet* m : s->gnets) mgnet_destroy(m);
    s->gnets.clear();
}

RTE_API rte_status rte_server_create_multi(const rte_server_config* cfg, mgnet* const* nets, int count,
                                           rte_server** out) {
    if (!cfg || !out || cfg->slots < 1 || cfg->slots > 64 || cfg->max_device_bytes == 0 || count < 0 ||
        count > 16 || (count > 0 && !nets)) {
        set_error(nullptr, "bad server configuration (slots in [1, 64], at most 16 networks)");
        return RTE_EINVAL;
    }
    *out = nullptr;
    std::vector<mgnet_config> ncfg;
    for (int k = 0; k < count; ++k) {
        mgnet_config c{};
        if (mgnet_get_config(nets[k], &c) != RTE_OK) return RTE_EINVAL;
        for (const mgnet_config& o : ncfg)
            if (o.M == c.M) {
                set_error(nullptr, "two networks for the same M");
                return RTE_EINVAL;
            }
        ncfg.push_back(c);
    }
    rte_server* s = new (std::nothrow) rte_server();
    if (!s) { set_error(nullptr, "host allocation failed"); return RTE_ENOMEM; }
    s->cfg = *cfg;
    s->net_cfg = ncfg;
    cudaGetDevice(&s->device);
    if (cfg->grouped) {
        if (cudaStreamCreateWithFlags(&s->gst, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            set_error(nullptr, "cudaStreamCreate failed");
            return RTE_ECUDA;
        }
        for (int k = 0; k < count; ++k) {
            mgnet* c = nullptr;
            rte_status st = mgnet_clone(nets[k], s->gst, &c);
            if (st != RTE_OK) {
                destroy_nets(s);
                cudaStreamDestroy(s->gst);
                delete s;
                return st;
            }
            s->gnets.push_back(c);
        }
        s->workers.emplace_back(admit_main, s);
        s->workers.emplace_back(setup_main, s);
        s->workers.emplace_back(setup_main, s);
        s->workers.emplace_back(group_main, s);
        *out = s;
        return RTE_OK;
    }
    s->nets.resize(cfg->slots);
    for (int i = 0; i < cfg->slots; ++i)
        for (int k = 0; k < count; ++k) {
            mgnet* c = nullptr;
            rte_status st = mgnet_clone(nets[k], nullptr, &c);
            if (st != RTE_OK) {
                destroy_nets(s);
                delete s;
                return st;
            }
            s->nets[i].push_back(c);
        }
    for (int i = 0; i < cfg->slots; ++i) s->workers.emplace_back(worker_main, s, i);
    *out = s;
    return RTE_OK;
}

RTE_API rte_status rte_server_create(const rte_server_config* cfg, mgnet* net, rte_server** out) {
    return rte_server_create_multi(cfg, net ? &net : nullptr, net ? 1 : 0, out);
}

RTE_API rte_status rte_server_submit(rte_server* s, const rte_request* r, int64_t* id_out) {
    if (!s || !r || !id_out) { set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    std::string why;
    if (!valid_request(r, why)) { set_error(nullptr, "malformed request: " + why); return RTE_EINVAL; }
    auto job = std::make_shared<Job>();
    const size_t N = (size_t)r->I * r->I;
    job->I = r->I;
    job->M = r->M;
    job->sT.assign(r->sigma_T, r->sigma_T + N);
    job->sa.assign(r->sigma_a, r->sigma_a + N);
    job->q.assign(r->q, r->q + N);
    job->eps_is_scalar = r->eps_is_scalar;
    job->eps.assign(r->eps, r->eps + (r->eps_is_scalar ? 1 : N));
    if (r->inflow) job->inflow.assign(r->inflow, r->inflow + (size_t)4 * r->I * r->M);
    job->g = r->g;
    rte_solve_opts_default(&job->opts);
    job->opts.tol = r->tol > 0 ? r->tol : 1e-8;
    if (r->max_iter > 0) job->opts.max_iter = r->max_iter;
    if (r->restart > 0) job->opts.restart = r->restart;
    job->net = r->use_net ? pick_net(s, r->I, r->M) : -1;
    job->use_net = job->net >= 0;
    job->footprint = footprint(r->I, r->M, job->opts.restart, job->use_net, count_materials(*job));
    if (job->footprint > s->cfg.max_device_bytes) {
        set_error(nullptr, "request needs more device memory than the server budget");
        return RTE_ENOMEM;
    }
    job->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) { set_error(nullptr, "server is stopping"); return RTE_ECANCELLED; }
        job->id = s->next_id++;
        s->jobs[job->id] = job;
        s->queue.push_back(job);
    }
    s->cv_work.notify_all();
    *id_out = job->id;
    return RTE_OK;
}

static void fill_result(const Job& j, rte_result* res, double* psi_host) {
    if (res) {
        res->status = j.status;
        res->info = j.info;
        res->latency_s = std::chrono::duration<double>(j.t_end - j.t_submit).count();
        res->queue_s = std::chrono::duration<double>(j.t_start - j.t_submit).count();
        res->footprint = j.footprint;
        res->used_net = j.use_net;
    }
    if (psi_host && !j.psi.empty()) std::memcpy(psi_host, j.psi.data(), j.psi.size() * sizeof(double));
}

RTE_API rte_status rte_server_wait(rte_server* s, int64_t id, double timeout_ms, rte_result* res,
                                   double* psi_host) {
    if (!s) { set_error(nullptr, "NULL server"); return RTE_EINVAL; }
    std::shared_ptr<Job> job;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->jobs.find(id);
        if (it == s->jobs.end()) { set_error(nullptr, "unknown request id"); return RTE_EINVAL; }
        job = it->second;
        auto pred = [&] { return job->done; };
        if (timeout_ms > 0) {
            if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred))
                return RTE_ETIMEOUT;
        } else {
            s->cv_done.wait(lk, pred);
        }
        s->jobs.erase(id);
    }
    fill_result(*job, res, psi_host);
    if (job->status != RTE_OK) set_error(nullptr, job->err);
    return RTE_OK;
}

RTE_API rte_status rte_server_cancel(rte_server* s, int64_t id) {
    if (!s) { set_error(nullptr, "NULL server"); return RTE_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) { set_error(nullptr, "unknown request id"); return RTE_EINVAL; }
    it->second->cancel = 1;
    s->cv_work.notify_all();
    return RTE_OK;
}

RTE_API rte_status rte_server_stats(rte_server* s, rte_server_stats_t* st) {
    if (!s || !st) { set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    st->queued = (int64_t)s->queue.size();
    st->active = s->active;
    st->completed = s->completed;
    st->bytes_in_use = s->bytes_in_use;
    return RTE_OK;
}

RTE_API void rte_server_destroy(rte_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        for (auto& kv : s->jobs) kv.second->cancel = 1;
    }
    s->cv_work.notify_all();
    s->cv_setup.notify_all();
    s->cv_group.notify_all();
    for (auto& t : s->workers) t.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& j : s->queue) {
            j->status = RTE_ECANCELLED;
            j->done = true;
        }
    }
    s->cv_done.notify_all();
    {
        // grouped mode: requests set up but never run
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& j : s->ready) {
            if (j->x) cudaFreeAsync(j->x, s->gst);
            if (j->psi_dev) cudaFreeAsync(j->psi_dev, s->gst);
            if (j->ctx) rte_destroy(j->ctx);
            j->status = RTE_ECANCELLED;
            j->done = true;
        }
        for (auto& j : s->setup_q) {
            j->status = RTE_ECANCELLED;
            j->done = true;
        }
    }
    s->cv_done.notify_all();
    destroy_nets(s);
    if (s->gst) {
        cudaStreamSynchronize(s->gst);
        cudaStreamDestroy(s->gst);
    }
    delete s;
}

}  // extern "C"
