// Continuous-batching scoring server.
//
// The paper scores poses in fixed batches per rank and writes results only at
// job end (Section 4.2), noting that results should rather be written as they
// are computed.  Here a request loop takes poses one by one as they arrive and
// scores them in batches on the GPU:
//
//  * a slot is a model replica with its own device workspace and stream; the
//    number of slots is admitted against an HBM budget (each slot's footprint
//    is measured when the first one is created);
//  * one worker thread per slot takes whatever poses are queued (waiting at
//    most a batching window for the batch to fill), packs them into pinned
//    host memory and scores them; while one slot's batch runs on the GPU the
//    others take the requests that arrived meanwhile, so batches overlap on the
//    device and no request waits for a full drain;
//  * a pose's result is available as soon as its batch completes, with its
//    latency from submission to completion.
//
// Scoring a pose does not depend on the other poses of its batch (every kernel
// reduces in a fixed per-pose order and FP8 scales are per pose), so a result
// is the same whether the pose was scored alone or in any mix.
#include "fusion_internal.cuh"

#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    int32_t n_atoms, n_lig;
    std::vector<float> xyz, feat;
    Clock::time_point t_arrive;
};

struct Result {
    float affinity;
    double latency_s;
    int status;
};

struct Slot {
    fusion_model *model = nullptr;
    int32_t *off = nullptr, *nlig = nullptr;
    float *xyz = nullptr, *feat = nullptr, *out = nullptr;
};

}  // namespace

struct fusion_server {
    fusion_server_config cfg{};
    int device = 0;
    int32_t max_atoms = 0;
    size_t slot_bytes = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Result> done;
    std::unordered_set<uint64_t> outstanding;   // submitted, result not yet collected
    uint64_t next_ticket = 1;
    int64_t inflight = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    // statistics
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, failed = 0;
    double gpu_busy_s = 0.0;
};

namespace {

void worker_loop(fusion_server *s, int si) {
    cudaSetDevice(s->device);
    Slot &sl = s->slots[si];
    std::vector<Request> batch;
    batch.reserve(s->cfg.max_batch);
    const auto window = std::chrono::duration<double, std::micro>(s->cfg.batch_window_us);
    while (true) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            if (s->queue.empty()) break;   // stop requested and nothing left
            const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(window);
            while ((int)s->queue.size() < s->cfg.max_batch && !s->stop) {
                if (s->cv_work.wait_until(lk, deadline) == std::cv_status::timeout) break;
            }
            if (s->queue.empty()) continue;    // another slot took them
            const int k = std::min<int>(s->cfg.max_batch, (int)s->queue.size());
            batch.clear();
            for (int i = 0; i < k; ++i) {
                batch.push_back(std::move(s->queue.front()));
                s->queue.pop_front();
            }
            s->inflight += k;
        }
        const int k = (int)batch.size();
        sl.off[0] = 0;
        for (int i = 0; i < k; ++i) {
            const Request &r = batch[i];
            sl.off[i + 1] = sl.off[i] + r.n_atoms;
            sl.nlig[i] = r.n_lig;
            std::memcpy(sl.xyz + (size_t)sl.off[i] * 3, r.xyz.data(), sizeof(float) * 3 * r.n_atoms);
            std::memcpy(sl.feat + (size_t)sl.off[i] * 19, r.feat.data(), sizeof(float) * 19 * r.n_atoms);
        }
        fusion_poses p{k, sl.off, sl.nlig, sl.xyz, sl.feat, 0};
        const auto t0 = Clock::now();
        const int rc = fusion_score(sl.model, &p, k, sl.out);
        const auto t1 = Clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (int i = 0; i < k; ++i) {
                const double lat = std::chrono::duration<double>(t1 - batch[i].t_arrive).count();
                s->done[batch[i].ticket] = Result{rc == FUSION_OK ? sl.out[i] : NAN, lat, rc};
            }
            s->inflight -= k;
            s->completed += k;
            s->batches += 1;
            if (rc != FUSION_OK) s->failed += k;
            s->gpu_busy_s += std::chrono::duration<double>(t1 - t0).count();
        }
        s->cv_done.notify_all();
    }
}

int srv_fail(int code, const std::string &m) { return fusion::set_last_error(code, m.c_str()); }

}  // namespace

extern "C" {

int fusion_server_create(const fusion_model_desc *desc, const void *weights, size_t weights_bytes,
                         const fusion_server_config *cfg, fusion_server **out) {
    if (!desc || !cfg || !out) return srv_fail(FUSION_EINVAL, "NULL argument");
    if (cfg->max_batch < 1 || cfg->max_batch > desc->max_poses)
        return srv_fail(FUSION_EINVAL, "max_batch must be in [1, desc->max_poses]");
    if (cfg->slots < 0 || cfg->slots > 16) return srv_fail(FUSION_EINVAL, "slots must be in [0, 16]");
    if (cfg->queue_capacity < 1) return srv_fail(FUSION_EINVAL, "queue_capacity must be >= 1");
    if (!(cfg->batch_window_us >= 0.0)) return srv_fail(FUSION_EINVAL, "batch_window_us must be >= 0");
    fusion_server *s = new fusion_server();
    s->cfg = *cfg;
    s->max_atoms = desc->max_atoms;
    cudaGetDevice(&s->device);
    fusion_model_desc d = *desc;
    d.max_poses = cfg->max_batch;
    const int want = cfg->slots > 0 ? cfg->slots : 4;
    for (int i = 0; i < want; ++i) {
        // HBM budget admission: a further slot is created only if all slots fit the budget
        if (cfg->hbm_budget_bytes > 0 && i > 0 && (size_t)(i + 1) * s->slot_bytes > cfg->hbm_budget_bytes) break;
        size_t free0 = 0, free1 = 0, total = 0;
        cudaMemGetInfo(&free0, &total);
        Slot sl;
        int rc = fusion_create(&d, weights, weights_bytes, nullptr, &sl.model);
        if (rc) {
            if (i == 0) {
                delete s;
                return rc;
            }
            break;   // no memory for more slots: serve with the ones admitted
        }
        cudaMemGetInfo(&free1, &total);
        if (i == 0) {
            s->slot_bytes = free0 > free1 ? free0 - free1 : 0;
            if (cfg->hbm_budget_bytes > 0 && s->slot_bytes > cfg->hbm_budget_bytes) {
                const size_t need = s->slot_bytes;
                fusion_destroy(sl.model);
                delete s;
                return srv_fail(FUSION_ENOMEM, "one slot (" + std::to_string(need) + " bytes) exceeds the HBM budget");
            }
        }
        const size_t A = (size_t)cfg->max_batch * desc->max_atoms;
        if (cudaMallocHost(&sl.off, sizeof(int32_t) * (cfg->max_batch + 1)) != cudaSuccess ||
            cudaMallocHost(&sl.nlig, sizeof(int32_t) * cfg->max_batch) != cudaSuccess ||
            cudaMallocHost(&sl.xyz, sizeof(float) * A * 3) != cudaSuccess ||
            cudaMallocHost(&sl.feat, sizeof(float) * A * 19) != cudaSuccess ||
            cudaMallocHost(&sl.out, sizeof(float) * cfg->max_batch) != cudaSuccess) {
            fusion_destroy(sl.model);
            cudaGetLastError();
            if (i == 0) {
                delete s;
                return srv_fail(FUSION_ENOMEM, "pinned host buffers for a slot");
            }
            break;
        }
        s->slots.push_back(sl);
    }
    for (int i = 0; i < (int)s->slots.size(); ++i) s->workers.emplace_back(worker_loop, s, i);
    *out = s;
    return FUSION_OK;
}

int fusion_server_submit(fusion_server *s, const float *xyz, const float *feat, int32_t n_atoms, int32_t n_lig,
                         uint64_t *ticket) {
    if (!s || !xyz || !feat || !ticket) return srv_fail(FUSION_EINVAL, "NULL argument");
    if (n_atoms < 1 || n_atoms > s->max_atoms) return srv_fail(FUSION_EINVAL, "n_atoms outside [1, max_atoms]");
    if (n_lig < 1 || n_lig > n_atoms) return srv_fail(FUSION_EINVAL, "n_lig outside [1, n_atoms]");
    for (int i = 0; i < 3 * n_atoms; ++i)
        if (!std::isfinite(xyz[i])) return srv_fail(FUSION_EINVAL, "non-finite coordinate");
    Request r;
    r.n_atoms = n_atoms;
    r.n_lig = n_lig;
    r.xyz.assign(xyz, xyz + 3 * n_atoms);
    r.feat.assign(feat, feat + 19 * n_atoms);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return srv_fail(FUSION_EINVAL, "server is shutting down");
        if ((int64_t)s->queue.size() >= s->cfg.queue_capacity) {
            s->rejected += 1;
            return srv_fail(FUSION_EAGAIN, "queue full");
        }
        r.ticket = s->next_ticket++;
        r.t_arrive = Clock::now();
        *ticket = r.ticket;
        s->outstanding.insert(r.ticket);
        s->queue.push_back(std::move(r));
        s->submitted += 1;
    }
    s->cv_work.notify_one();
    return FUSION_OK;
}

int fusion_server_poll(fusion_server *s, uint64_t ticket, float *affinity, double *latency_s) {
    if (!s) return srv_fail(FUSION_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        if (ticket == 0 || ticket >= s->next_ticket) return srv_fail(FUSION_EINVAL, "unknown ticket");
        if (!s->outstanding.count(ticket)) return srv_fail(FUSION_EINVAL, "ticket already collected");
        return FUSION_EAGAIN;
    }
    const Result r = it->second;
    s->done.erase(it);
    s->outstanding.erase(ticket);
    if (affinity) *affinity = r.affinity;
    if (latency_s) *latency_s = r.latency_s;
    if (r.status != FUSION_OK) return srv_fail(r.status, "scoring the batch of this pose failed");
    return FUSION_OK;
}

int fusion_server_drain(fusion_server *s, double timeout_s) {
    if (!s) return srv_fail(FUSION_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    const bool ok = s->cv_done.wait_until(lk, until, [&] { return s->queue.empty() && s->inflight == 0; });
    return ok ? FUSION_OK : srv_fail(FUSION_ETIMEOUT, "drain timed out");
}

int fusion_server_get_stats(fusion_server *s, fusion_server_stats *st) {
    if (!s || !st) return srv_fail(FUSION_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    st->slots = (int32_t)s->slots.size();
    st->slot_bytes = s->slot_bytes;
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->failed = s->failed;
    st->batches = s->batches;
    st->queued = (int64_t)s->queue.size();
    st->inflight = s->inflight;
    st->gpu_busy_s = s->gpu_busy_s;
    return FUSION_OK;
}

void fusion_server_destroy(fusion_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto &sl : s->slots) {
        fusion_destroy(sl.model);
        cudaFreeHost(sl.off);
        cudaFreeHost(sl.nlig);
        cudaFreeHost(sl.xyz);
        cudaFreeHost(sl.feat);
        cudaFreeHost(sl.out);
    }
    delete s;
}

}  // extern "C"
