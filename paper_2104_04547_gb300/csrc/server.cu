// Continuous-batching scoring server.
//
// The paper scores poses in fixed batches per rank and writes results only at
// job end (Section 4.2), noting that results should rather be written as they
// are computed.  Here a request loop takes poses one by one as they arrive and
// scores them in batches on the GPU:
//
//  * a slot is a model replica with its own device workspace and stream; the
//    number of slots is admitted against an HBM budget (each dtype's slot
//    footprint is measured when its first slot is created);
//  * one server may run slots of several conv dtypes (BF16 and FP8): each
//    request names its dtype (or takes the descriptor's), waits in that
//    dtype's queue and is scored by a slot of that dtype;
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
#include <algorithm>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kDtypes = 3;   // FUSION_F32, FUSION_BF16, FUSION_FP8

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
    int dtype = 0;
    fusion_model *model = nullptr;
    int32_t *off = nullptr, *nlig = nullptr;
    float *xyz = nullptr, *feat = nullptr, *out = nullptr;
};

}  // namespace

struct fusion_server {
    fusion_server_config cfg{};
    int device = 0;
    int32_t max_atoms = 0;
    int default_dtype = 0;
    unsigned dtype_mask = 0;                     // dtypes this server has slots for
    size_t slot_bytes = 0;                       // largest measured slot footprint
    size_t dtype_bytes[kDtypes] = {};            // measured footprint of one slot of each dtype
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work[kDtypes], cv_done;
    std::deque<Request> queue[kDtypes];          // one queue per dtype
    int64_t queued_total = 0;
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
    std::deque<Request> &q = s->queue[sl.dtype];
    std::condition_variable &cv = s->cv_work[sl.dtype];
    std::vector<Request> batch;
    batch.reserve(s->cfg.max_batch);
    const auto window = std::chrono::duration<double, std::micro>(s->cfg.batch_window_us);
    while (true) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            cv.wait(lk, [&] { return s->stop || !q.empty(); });
            if (q.empty()) break;   // stop requested and nothing left
            const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(window);
            while ((int)q.size() < s->cfg.max_batch && !s->stop) {
                if (cv.wait_until(lk, deadline) == std::cv_status::timeout) break;
            }
            if (q.empty()) continue;    // another slot of this dtype took them
            const int k = std::min<int>(s->cfg.max_batch, (int)q.size());
            batch.clear();
            for (int i = 0; i < k; ++i) {
                batch.push_back(std::move(q.front()));
                q.pop_front();
            }
            s->queued_total -= k;
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
    if (cfg->dtypes & ~7u) return srv_fail(FUSION_EINVAL, "dtypes must be a mask of (1 << FUSION_F32/BF16/FP8)");
    if (desc->dtype < 0 || desc->dtype >= kDtypes) return srv_fail(FUSION_EINVAL, "bad dtype");
    fusion_server *s = new fusion_server();
    s->cfg = *cfg;
    s->max_atoms = desc->max_atoms;
    s->default_dtype = desc->dtype;
    s->dtype_mask = (unsigned)cfg->dtypes | (1u << desc->dtype);
    int dts[kDtypes], ndt = 0;
    for (int t = 0; t < kDtypes; ++t)
        if (s->dtype_mask & (1u << t)) dts[ndt++] = t;
    cudaGetDevice(&s->device);
    fusion_model_desc d = *desc;
    d.max_poses = cfg->max_batch;
    const int want = std::max(cfg->slots > 0 ? cfg->slots : 4, ndt);
    size_t used = 0;
    for (int i = 0; i < want; ++i) {
        // slots cycle through the dtypes; HBM budget admission: a further slot is created only if all slots
        // fit the budget (a dtype's footprint is measured on its first slot)
        const int dt = dts[i % ndt];
        const bool first_of_dtype = i < ndt;
        if (cfg->hbm_budget_bytes > 0 && !first_of_dtype && used + s->dtype_bytes[dt] > cfg->hbm_budget_bytes) break;
        size_t free0 = 0, free1 = 0, total = 0;
        cudaMemGetInfo(&free0, &total);
        Slot sl;
        sl.dtype = dt;
        d.dtype = dt;
        int rc = fusion_create(&d, weights, weights_bytes, nullptr, &sl.model);
        if (rc) {
            if (first_of_dtype) {
                fusion_server_destroy(s);
                return rc;
            }
            break;   // no memory for more slots: serve with the ones admitted
        }
        cudaMemGetInfo(&free1, &total);
        if (first_of_dtype) {
            s->dtype_bytes[dt] = free0 > free1 ? free0 - free1 : 0;
            s->slot_bytes = std::max(s->slot_bytes, s->dtype_bytes[dt]);
            if (cfg->hbm_budget_bytes > 0 && used + s->dtype_bytes[dt] > cfg->hbm_budget_bytes) {
                const size_t need = s->dtype_bytes[dt];
                fusion_destroy(sl.model);
                fusion_server_destroy(s);
                return srv_fail(FUSION_ENOMEM, "one slot (" + std::to_string(need) + " bytes) exceeds the HBM budget");
            }
        }
        used += s->dtype_bytes[dt];
        const size_t A = (size_t)cfg->max_batch * desc->max_atoms;
        if (cudaMallocHost(&sl.off, sizeof(int32_t) * (cfg->max_batch + 1)) != cudaSuccess ||
            cudaMallocHost(&sl.nlig, sizeof(int32_t) * cfg->max_batch) != cudaSuccess ||
            cudaMallocHost(&sl.xyz, sizeof(float) * A * 3) != cudaSuccess ||
            cudaMallocHost(&sl.feat, sizeof(float) * A * 19) != cudaSuccess ||
            cudaMallocHost(&sl.out, sizeof(float) * cfg->max_batch) != cudaSuccess) {
            fusion_destroy(sl.model);
            cudaFreeHost(sl.off);
            cudaFreeHost(sl.nlig);
            cudaFreeHost(sl.xyz);
            cudaFreeHost(sl.feat);
            cudaFreeHost(sl.out);
            cudaGetLastError();
            if (first_of_dtype) {
                fusion_server_destroy(s);
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
    if (!s) return srv_fail(FUSION_EINVAL, "NULL argument");
    return fusion_server_submit_dtype(s, xyz, feat, n_atoms, n_lig, s->default_dtype, ticket);
}

int fusion_server_submit_dtype(fusion_server *s, const float *xyz, const float *feat, int32_t n_atoms,
                               int32_t n_lig, int32_t dtype, uint64_t *ticket) {
    if (!s || !xyz || !feat || !ticket) return srv_fail(FUSION_EINVAL, "NULL argument");
    if (dtype < 0 || dtype >= kDtypes || !(s->dtype_mask & (1u << dtype)))
        return srv_fail(FUSION_EINVAL, "the server has no slots of this dtype");
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
        if (s->queued_total >= s->cfg.queue_capacity) {
            s->rejected += 1;
            return srv_fail(FUSION_EAGAIN, "queue full");
        }
        r.ticket = s->next_ticket++;
        r.t_arrive = Clock::now();
        *ticket = r.ticket;
        s->outstanding.insert(r.ticket);
        s->queue[dtype].push_back(std::move(r));
        s->queued_total += 1;
        s->submitted += 1;
    }
    s->cv_work[dtype].notify_one();
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
    const bool ok = s->cv_done.wait_until(lk, until, [&] { return s->queued_total == 0 && s->inflight == 0; });
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
    st->queued = s->queued_total;
    st->inflight = s->inflight;
    st->gpu_busy_s = s->gpu_busy_s;
    for (int t = 0; t < kDtypes; ++t) st->slots_by_dtype[t] = 0;
    for (const Slot &sl : s->slots) st->slots_by_dtype[sl.dtype] += 1;
    return FUSION_OK;
}

void fusion_server_destroy(fusion_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    for (auto &cv : s->cv_work) cv.notify_all();
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
