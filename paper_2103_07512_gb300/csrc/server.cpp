// server.cpp -- serving loop: evaluation jobs arrive over time, are admitted
// by device memory, fused (per domain into populations, across domains into
// one interpreter launch) and run on several streams at once.
//
// Threads and locks.  Callers submit and wait; one worker thread admits and
// launches; a CUDA host function enqueued after each launch's result copy
// completes its jobs.  srv->mu guards all server state.  The worker never
// makes a CUDA or context call while holding srv->mu, because such a call may
// wait for the device (an implicit or explicit synchronisation) and the host
// functions it would wait for take srv->mu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/tgp.h"
#include "compiler.h"
#include "internal.h"

namespace tgp {
namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

uint32_t bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

// Identity of a domain: grid, bounds and target.
struct DomainKey {
    int32_t W = 0, H = 0;
    uint32_t b[4] = {0, 0, 0, 0};
    int32_t kind = TGP_TARGET_PAGIE;
    int32_t order = 0;
    std::vector<int32_t> ops;    // target tree (TGP_TARGET_TOKENS)
    std::vector<float> imm;
    bool operator<(const DomainKey& o) const {
        if (W != o.W) return W < o.W;
        if (H != o.H) return H < o.H;
        for (int i = 0; i < 4; ++i)
            if (b[i] != o.b[i]) return b[i] < o.b[i];
        if (kind != o.kind) return kind < o.kind;
        if (order != o.order) return order < o.order;
        if (ops != o.ops) return ops < o.ops;
        if (imm.size() != o.imm.size()) return imm.size() < o.imm.size();
        for (size_t i = 0; i < imm.size(); ++i)
            if (bits(imm[i]) != bits(o.imm[i])) return bits(imm[i]) < bits(o.imm[i]);
        return false;
    }
    int64_t N() const { return (int64_t)W * H; }
};

struct Resident {
    tgp_handle h = 0;       // 0 while its first launch is loading it
    int64_t bytes = 0;
    int64_t last_use = 0;
    int in_use = 0;         // launches in flight on it
};

struct Job {
    int64_t id = 0;
    PopIR ir;
    int32_t n_trees = 0;
    DomainKey key;
    int64_t est = 0;                  // launch bytes
    int64_t dom_bytes = 0;            // bytes of its domain when resident
    std::shared_ptr<internal::PrePlan> plan;   // planned at submit (used when it runs alone)
    bool done = false;
    std::vector<double> rmse;
    tgp_job_info info{};
};

// Domains one fused launch may span at most.
constexpr int kMaxSegments = 64;

// One domain of a launch: its resident entry and the batch's jobs on it.
struct Segment {
    DomainKey key;
    Resident* dom = nullptr;
    bool load = false;   // the launch loads the domain first
    std::vector<Job*> jobs;
};

struct Slot {
    tgp_server* srv = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<tgp_handle> pops;   // one population per segment, kept for their buffers
    double* d_rmse = nullptr;
    double* h_rmse = nullptr;
    size_t cap = 0;
    SegParams* d_segs = nullptr;    // segment table of a fused launch
    int32_t* d_counter = nullptr;   // its work-queue heads
    bool busy = false;
    std::vector<Job*> jobs;         // segment by segment
    std::vector<Resident*> doms;
    int64_t bytes = 0;
};

}  // namespace
}  // namespace tgp

struct tgp_server {
    tgp_ctx* ctx = nullptr;
    int device = 0;
    tgp_server_config cfg{};
    std::mutex mu;
    std::condition_variable wake;   // worker: a job arrived, a slot freed, stop
    std::condition_variable done;   // waiters: a job finished
    bool stop = false;
    std::thread worker;
    int64_t next_id = 1;
    int64_t tick = 0;
    std::deque<tgp::Job*> pending;
    std::unordered_map<int64_t, std::unique_ptr<tgp::Job>> jobs;
    std::map<tgp::DomainKey, tgp::Resident> domains;
    std::vector<std::unique_ptr<tgp::Slot>> slots;
    int in_flight = 0;
    tgp_server_stats st{};
};

namespace tgp {
namespace {

#define SRV_TRY(call)                                                                               \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return internal::set_error(TGP_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Completes the jobs of a finished launch (host function on the slot's
// stream, after the result copy).  Makes no CUDA call.
void CUDART_CB on_launch_done(void* arg) {
    Slot* s = static_cast<Slot*>(arg);
    tgp_server* srv = s->srv;
    std::lock_guard<std::mutex> g(srv->mu);
    const int64_t t = now_ns();
    size_t off = 0;
    for (Job* j : s->jobs) {
        j->rmse.assign(s->h_rmse + off, s->h_rmse + off + j->n_trees);
        off += (size_t)j->n_trees;
        j->info.done_ns = t;
        j->info.status = TGP_OK;
        j->done = true;
        srv->st.completed++;
    }
    s->jobs.clear();
    s->busy = false;
    const int64_t tick = ++srv->tick;
    for (Resident* r : s->doms) {
        r->in_use--;
        r->last_use = tick;
    }
    s->doms.clear();
    srv->st.bytes_in_use -= s->bytes;
    s->bytes = 0;
    srv->in_flight--;
    srv->wake.notify_all();
    srv->done.notify_all();
}

// Marks the jobs of a launch that could not be enqueued as failed (lock held).
void fail_jobs(tgp_server* srv, Slot* s, int rc) {
    const int64_t t = now_ns();
    for (Job* j : s->jobs) {
        j->rmse.assign((size_t)j->n_trees, std::nan(""));
        j->info.done_ns = t;
        j->info.status = rc;
        j->done = true;
        srv->st.failed++;
    }
    s->jobs.clear();
    s->busy = false;
    for (Resident* r : s->doms) r->in_use--;
    s->doms.clear();
    srv->st.bytes_in_use -= s->bytes;
    s->bytes = 0;
    srv->in_flight--;
    srv->done.notify_all();
}

// Enqueues one launch: loads the segments' domains that are not resident,
// merges each segment's jobs into one population, runs the fitness of all
// segments (one fused interpreter launch when there are several) and copies
// the RMSE values back.  Called by the worker without srv->mu.
int launch(tgp_server* srv, Slot* s, std::vector<Segment>& segs) {
    tgp_ctx* ctx = srv->ctx;
    SRV_TRY(cudaSetDevice(srv->device));
    for (Segment& sg : segs) {
        if (!sg.load) continue;
        const DomainKey& key = sg.key;
        tgp_target_tokens tt{};
        const void* target = nullptr;
        if (key.kind == TGP_TARGET_TOKENS) {
            tt.ops = key.ops.data();
            tt.imm = key.imm.empty() ? nullptr : key.imm.data();
            tt.n_ops = (int64_t)key.ops.size();
            tt.n_imm = (int64_t)key.imm.size();
            tt.order = key.order;
            target = &tt;
        }
        float bd[4];
        std::memcpy(bd, key.b, sizeof bd);
        tgp_handle h = 0;
        const int64_t t0 = now_ns();
        int rc = internal::load_domain(ctx, key.W, key.H, bd[0], bd[1], bd[2], bd[3], key.kind, target, s->stream,
                                       false, &h);
        if (rc) return rc;
        std::lock_guard<std::mutex> g(srv->mu);
        sg.dom->h = h;
        srv->st.domains_loaded++;
        srv->st.domain_load_ns += now_ns() - t0;
    }
    size_t T = 0;
    for (const Segment& sg : segs)
        for (const Job* j : sg.jobs) T += (size_t)j->n_trees;
    if (T > s->cap) {
        if (s->d_rmse) cudaFree(s->d_rmse);
        if (s->h_rmse) cudaFreeHost(s->h_rmse);
        s->d_rmse = nullptr;
        s->h_rmse = nullptr;
        s->cap = 0;
        SRV_TRY(cudaMalloc(&s->d_rmse, T * sizeof(double)));
        SRV_TRY(cudaMallocHost(&s->h_rmse, T * sizeof(double)));
        s->cap = T;
    }
    std::vector<internal::FusedSegment> fused;
    size_t off = 0;
    const int64_t t_adopt = now_ns();
    for (size_t i = 0; i < segs.size(); ++i) {
        Segment& sg = segs[i];
        PopIR ir;
        std::shared_ptr<internal::PrePlan> pre;
        if (sg.jobs.size() == 1) {
            ir = std::move(sg.jobs[0]->ir);
            pre = std::move(sg.jobs[0]->plan);
        } else {
            for (Job* j : sg.jobs) {
                append_population(ir, j->ir);
                j->ir = PopIR();
                j->plan.reset();
            }
        }
        const size_t nt = ir.roots.size();
        if (i == s->pops.size()) s->pops.push_back(0);
        int rc = s->pops[i] ? internal::replace_population(ctx, s->pops[i], std::move(ir), std::move(pre))
                            : internal::adopt_population(ctx, std::move(ir), &s->pops[i], std::move(pre));
        if (rc) return rc;
        fused.push_back(internal::FusedSegment{s->pops[i], sg.dom->h, s->d_rmse + off});
        off += nt;
    }
    const int64_t t = now_ns();
    for (const Segment& sg : segs)
        for (Job* j : sg.jobs) j->info.launch_ns = t;
    int rc = segs.size() == 1 ? tgp_fitness_dev(ctx, fused[0].pop, fused[0].domain, s->stream, s->d_rmse)
                              : internal::fitness_fused(ctx, fused, s->stream, s->d_segs, s->d_counter);
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->st.adopt_ns += t - t_adopt;
        srv->st.fitness_ns += now_ns() - t;
    }
    if (rc) return rc;
    SRV_TRY(cudaMemcpyAsync(s->h_rmse, s->d_rmse, T * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SRV_TRY(cudaLaunchHostFunc(s->stream, on_launch_done, s));
    return TGP_OK;
}

// Resident domains kept at most; beyond it the least recently used idle ones
// are released in one batch down to the low mark (a release waits for the
// device, so it is done rarely).
constexpr size_t kMaxResidentDomains = 1024, kResidentLowMark = 768;

// Releases idle resident domains, least recently used first, until at most
// `keep` remain or `need` more bytes fit the budget (lock held on entry and
// exit, dropped around the releases).  Returns whether anything was released.
bool release_idle_domains(tgp_server* srv, std::unique_lock<std::mutex>& lk, size_t keep, int64_t need,
                          const DomainKey* spare) {
    std::vector<std::pair<int64_t, const DomainKey*>> lru;
    for (auto& kv : srv->domains)
        if (kv.second.in_use == 0 && kv.second.h != 0 && !(spare && !(kv.first < *spare) && !(*spare < kv.first)))
            lru.push_back({kv.second.last_use, &kv.first});
    std::sort(lru.begin(), lru.end());
    std::vector<tgp_handle> drop;
    for (auto& v : lru) {
        if (srv->domains.size() <= keep && srv->st.bytes_in_use + need <= srv->cfg.hbm_budget_bytes) break;
        auto it = srv->domains.find(*v.second);
        srv->st.bytes_in_use -= it->second.bytes;
        drop.push_back(it->second.h);
        srv->domains.erase(it);
        srv->st.domains_released++;
    }
    srv->st.domains_resident = (int64_t)srv->domains.size();
    if (drop.empty()) return false;
    lk.unlock();
    for (tgp_handle h : drop) tgp_release_domain(srv->ctx, h);
    lk.lock();
    return true;
}

void worker_main(tgp_server* srv) {
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        Slot* slot = nullptr;
        for (auto& s : srv->slots)
            if (!s->busy) { slot = s.get(); break; }
        if (srv->stop && srv->pending.empty() && srv->in_flight == 0) break;
        if (!slot || srv->pending.empty()) {
            srv->wake.wait(lk);
            continue;
        }
        Job* head = srv->pending.front();
        const DomainKey& key = head->key;
        auto rit = srv->domains.find(key);
        const bool resident = rit != srv->domains.end();
        const int64_t budget = srv->cfg.hbm_budget_bytes;
        int64_t need = head->est + (resident ? 0 : head->dom_bytes);
        if (srv->st.bytes_in_use + need > budget) {
            // room by releasing resident domains no launch uses, least recently used first
            int64_t freeable = 0;
            for (auto& kv : srv->domains)
                if (kv.second.in_use == 0 && kv.second.h != 0 && !(resident && &kv.second == &rit->second))
                    freeable += kv.second.bytes;
            if (srv->st.bytes_in_use - freeable + need > budget) {
                if (srv->in_flight > 0) {   // wait for launches to finish
                    srv->wake.wait(lk);
                    continue;
                }
                // nothing runs and it still does not fit: the job cannot run
                srv->pending.pop_front();
                head->rmse.assign((size_t)head->n_trees, std::nan(""));
                head->info.done_ns = now_ns();
                head->info.status = TGP_E_BUDGET;
                head->done = true;
                srv->st.failed++;
                srv->done.notify_all();
                continue;
            }
            const DomainKey kc = key;
            release_idle_domains(srv, lk, SIZE_MAX, need, resident ? &kc : nullptr);
            continue;
        }
        if (!resident && srv->domains.size() >= kMaxResidentDomains) {
            if (release_idle_domains(srv, lk, kResidentLowMark, 0, nullptr)) continue;
        }
        // the batch: the head, every later queued job on the head's domain,
        // and queued jobs on other domains (resident, or loadable within the
        // budget) that plan to the head's launch shape -- one fused launch
        std::vector<Segment> segs(1);
        segs.reserve(kMaxSegments);
        segs[0].key = key;
        segs[0].jobs.push_back(head);
        int64_t trees = head->n_trees;
        int64_t bytes = need;
        const bool fusable = head->plan != nullptr;
        const int hK = fusable ? head->plan->shape.K : 0, hT = fusable ? head->plan->shape.threads : 0;
        for (auto it = std::next(srv->pending.begin()); it != srv->pending.end(); ++it) {
            Job* j = *it;
            if (trees + j->n_trees > srv->cfg.max_batch_trees) continue;
            Segment* sg = nullptr;
            for (Segment& x : segs)
                if (!(x.key < j->key) && !(j->key < x.key)) { sg = &x; break; }
            int64_t add = j->est;
            if (!sg) {
                if (!fusable || !j->plan || j->plan->shape.K != hK || j->plan->shape.threads != hT) continue;
                if ((int)segs.size() >= kMaxSegments) continue;
                auto jr = srv->domains.find(j->key);
                if (jr != srv->domains.end()) {
                    if (jr->second.h == 0) continue;   // being loaded by a launch in flight
                } else {
                    add += j->dom_bytes;
                }
            }
            if (srv->st.bytes_in_use + bytes + add > budget) continue;
            if (!sg) {
                segs.emplace_back();
                segs.back().key = j->key;
                sg = &segs.back();
            }
            sg->jobs.push_back(j);
            trees += j->n_trees;
            bytes += add;
        }
        size_t n_jobs = 0;
        for (Segment& sg : segs)
            for (Job* j : sg.jobs) {
                srv->pending.erase(std::find(srv->pending.begin(), srv->pending.end(), j));
                ++n_jobs;
            }
        int64_t dom_new = 0;   // bytes of the domains this launch loads
        slot->jobs.clear();
        slot->doms.clear();
        for (Segment& sg : segs) {
            auto dit = srv->domains.find(sg.key);
            if (dit == srv->domains.end()) {
                Resident& r = srv->domains[sg.key];
                r.bytes = sg.jobs[0]->dom_bytes;
                dom_new += r.bytes;
                sg.dom = &r;
                sg.load = true;
            } else {
                sg.dom = &dit->second;
            }
            sg.dom->in_use++;
            slot->doms.push_back(sg.dom);
            for (Job* j : sg.jobs) slot->jobs.push_back(j);
        }
        srv->st.domains_resident = (int64_t)srv->domains.size();
        slot->busy = true;
        slot->bytes = bytes - dom_new;
        srv->st.bytes_in_use += bytes;
        srv->st.max_bytes_in_use = std::max(srv->st.max_bytes_in_use, srv->st.bytes_in_use);
        const int64_t bno = srv->st.batches++;
        srv->st.max_batch_jobs = std::max<int64_t>(srv->st.max_batch_jobs, (int64_t)n_jobs);
        srv->st.max_batch_domains = std::max<int64_t>(srv->st.max_batch_domains, (int64_t)segs.size());
        srv->in_flight++;
        srv->st.max_in_flight = std::max<int64_t>(srv->st.max_in_flight, srv->in_flight);
        for (Job* j : slot->jobs) {
            j->info.batch = bno;
            j->info.batch_jobs = (int32_t)n_jobs;
        }
        lk.unlock();
        const int64_t t_busy = now_ns();
        int rc = launch(srv, slot, segs);
        if (rc) cudaStreamSynchronize(slot->stream);   // nothing of this launch still runs
        lk.lock();
        srv->st.worker_busy_ns += now_ns() - t_busy;
        if (rc) {
            fail_jobs(srv, slot, rc);   // drops the launch's uses and bytes
            for (Segment& sg : segs) {
                if (sg.load && sg.dom->h == 0) {   // the domain never loaded
                    srv->st.bytes_in_use -= sg.dom->bytes;
                    srv->domains.erase(sg.key);
                }
            }
            srv->st.domains_resident = (int64_t)srv->domains.size();
        }
    }
}

}  // namespace
}  // namespace tgp

using namespace tgp;

extern "C" {

int tgp_server_create(tgp_ctx* ctx, const tgp_server_config* cfg, tgp_server** out) {
    if (!ctx || !out) return internal::set_error(TGP_E_INVALID, "ctx / out is NULL");
    *out = nullptr;
    int rc = TGP_OK;
    std::unique_ptr<tgp_server> srv(new (std::nothrow) tgp_server());
    if (!srv) return internal::set_error(TGP_E_NOMEM, "out of host memory");
    srv->ctx = ctx;
    if (cfg) srv->cfg = *cfg;
    if (srv->cfg.streams == 0) srv->cfg.streams = 4;
    if (srv->cfg.streams < 1 || srv->cfg.streams > 16)
        return internal::set_error(TGP_E_INVALID, "streams must be 1..16 (got %d)", srv->cfg.streams);
    if (srv->cfg.max_batch_trees == 0) srv->cfg.max_batch_trees = 4096;
    if (srv->cfg.max_batch_trees < 1)
        return internal::set_error(TGP_E_INVALID, "max_batch_trees must be >= 1");
    if (srv->cfg.hbm_budget_bytes < 0) return internal::set_error(TGP_E_INVALID, "hbm_budget_bytes < 0");
    // the context's device (a host-only context cannot serve)
    rc = internal::context_device(ctx, &srv->device);
    if (rc) return rc;
    SRV_TRY(cudaSetDevice(srv->device));
    if (srv->cfg.hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        SRV_TRY(cudaMemGetInfo(&fr, &tot));
        srv->cfg.hbm_budget_bytes = (int64_t)(0.8 * (double)fr);
    }
    srv->st.hbm_budget_bytes = srv->cfg.hbm_budget_bytes;
    for (int i = 0; i < srv->cfg.streams; ++i) {
        auto s = std::make_unique<Slot>();
        s->srv = srv.get();
        SRV_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
        const size_t cap = (size_t)srv->cfg.max_batch_trees;
        SRV_TRY(cudaMalloc(&s->d_rmse, cap * sizeof(double)));
        SRV_TRY(cudaMallocHost(&s->h_rmse, cap * sizeof(double)));
        s->cap = cap;
        SRV_TRY(cudaMalloc(&s->d_segs, kMaxSegments * sizeof(SegParams)));
        SRV_TRY(cudaMalloc(&s->d_counter, kQueueWords * sizeof(int32_t)));
        srv->slots.push_back(std::move(s));
    }
    tgp_server* raw = srv.get();
    srv->worker = std::thread(worker_main, raw);
    *out = srv.release();
    return TGP_OK;
}

int tgp_server_destroy(tgp_server* srv) {
    if (!srv) return internal::set_error(TGP_E_INVALID, "srv is NULL");
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
    }
    srv->wake.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    cudaSetDevice(srv->device);
    for (auto& s : srv->slots) {
        if (s->stream) cudaStreamSynchronize(s->stream);
        for (tgp_handle p : s->pops)
            if (p) tgp_release_population(srv->ctx, p);
        if (s->stream) cudaStreamDestroy(s->stream);
        if (s->d_rmse) cudaFree(s->d_rmse);
        if (s->h_rmse) cudaFreeHost(s->h_rmse);
        if (s->d_segs) cudaFree(s->d_segs);
        if (s->d_counter) cudaFree(s->d_counter);
    }
    for (auto& kv : srv->domains)
        if (kv.second.h) tgp_release_domain(srv->ctx, kv.second.h);
    delete srv;
    return TGP_OK;
}

int tgp_server_submit(tgp_server* srv, const tgp_job* job, int64_t* job_id) {
    if (!srv || !job || !job_id) return internal::set_error(TGP_E_INVALID, "srv / job / job_id is NULL");
    const int64_t arrival = now_ns();   // validation and hash-consing count as service time
    if (job->W < 1 || job->H < 1 || (int64_t)job->W * job->H > INT32_MAX)
        return internal::set_error(TGP_E_INVALID, "grid %d x %d: need W, H >= 1 and W*H <= 2^31-1", job->W,
                                   job->H);
    if (!std::isfinite(job->xlo) || !std::isfinite(job->xhi) || !std::isfinite(job->ylo) ||
        !std::isfinite(job->yhi))
        return internal::set_error(TGP_E_INVALID, "domain bounds must be finite");
    auto j = std::make_unique<Job>();
    DomainKey key;
    key.W = job->W;
    key.H = job->H;
    key.b[0] = bits(job->xlo);
    key.b[1] = bits(job->xhi);
    key.b[2] = bits(job->ylo);
    key.b[3] = bits(job->yhi);
    key.kind = job->target_kind;
    std::string err;
    if (job->target_kind == TGP_TARGET_TOKENS) {
        const tgp_target_tokens* tt = job->target_tokens;
        if (!tt || !tt->ops || tt->n_ops < 1) return internal::set_error(TGP_E_INVALID, "target tokens are NULL");
        PopIR probe;
        int64_t off[2] = {0, tt->n_ops};
        int prc = parse_population(tt->ops, tt->imm, tt->n_imm, off, 1, tt->order, probe, err,
                                   internal::context_simplifies(srv->ctx));
        if (prc)
            return internal::set_error(prc == -2 ? TGP_E_TOKENS : TGP_E_INVALID, "target tree: %s", err.c_str());
        key.order = tt->order;
        key.ops.assign(tt->ops, tt->ops + tt->n_ops);
        if (tt->n_imm > 0) key.imm.assign(tt->imm, tt->imm + tt->n_imm);
    } else if (job->target_kind != TGP_TARGET_PAGIE) {
        return internal::set_error(TGP_E_INVALID, "a job's target is Pagie or one target tree (kind %d)",
                                   job->target_kind);
    }
    int prc = parse_population(job->ops, job->imm, job->n_imm, job->tree_off, job->n_trees, job->order, j->ir, err,
                               internal::context_simplifies(srv->ctx));
    if (prc) return internal::set_error(prc == -2 ? TGP_E_TOKENS : TGP_E_INVALID, "%s", err.c_str());
    j->n_trees = job->n_trees;
    j->est = internal::estimate_bytes(srv->ctx, j->ir, key.N(), key.W);
    // the bytecode is planned here, in the caller's thread, for a launch of
    // this job alone (a fused launch is planned again by the worker)
    internal::preplan(srv->ctx, j->ir, key.N(), key.W, &j->plan);
    // a token target's values, and the Pagie column table (x part per column)
    j->dom_bytes = (key.kind == TGP_TARGET_TOKENS ? key.N() * (int64_t)sizeof(float) : 0) +
                   (key.W + 15) / 16 * 16 * (int64_t)sizeof(float);
    if (j->est + j->dom_bytes > srv->cfg.hbm_budget_bytes)
        return internal::set_error(TGP_E_BUDGET, "job needs %lld bytes of device memory; the budget is %lld",
                                   (long long)(j->est + j->dom_bytes), (long long)srv->cfg.hbm_budget_bytes);
    j->key = std::move(key);
    std::lock_guard<std::mutex> g(srv->mu);
    if (srv->stop) return internal::set_error(TGP_E_BUSY, "server is shutting down");
    j->id = srv->next_id++;
    j->info.submit_ns = arrival;
    *job_id = j->id;
    srv->pending.push_back(j.get());
    srv->jobs[j->id] = std::move(j);
    srv->st.submitted++;
    srv->wake.notify_all();
    return TGP_OK;
}

int tgp_server_wait(tgp_server* srv, int64_t job_id, int64_t timeout_us, double* rmse_host, tgp_job_info* info) {
    if (!srv) return internal::set_error(TGP_E_INVALID, "srv is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return internal::set_error(TGP_E_INVALID, "unknown job id %lld", (long long)job_id);
    Job* j = it->second.get();
    auto ready = [&] { return j->done; };
    if (timeout_us < 0) {
        srv->done.wait(lk, ready);
    } else if (!srv->done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
        return internal::set_error(TGP_E_TIMEOUT, "job %lld not done within %lld us", (long long)job_id,
                                   (long long)timeout_us);
    }
    if (rmse_host) std::copy(j->rmse.begin(), j->rmse.end(), rmse_host);
    if (info) *info = j->info;
    const int status = j->info.status;
    srv->jobs.erase(it);
    if (status) return internal::set_error(status, "job %lld failed (status %d)", (long long)job_id, status);
    return TGP_OK;
}

int tgp_server_stats_get(tgp_server* srv, tgp_server_stats* out) {
    if (!srv || !out) return internal::set_error(TGP_E_INVALID, "srv / out is NULL");
    std::lock_guard<std::mutex> g(srv->mu);
    *out = srv->st;
    out->queued = (int64_t)srv->pending.size();
    out->domains_resident = (int64_t)srv->domains.size();
    return TGP_OK;
}

}  // extern "C"
