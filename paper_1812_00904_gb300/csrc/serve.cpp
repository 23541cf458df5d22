// Serving runtime: continuous batching of single products over many resident
// matrices.
//
// One scheduler thread owns the dispatch decisions.  Requests queue in arrival
// order.  Whenever a stream slot is free, the oldest waiting request whose
// matrix is resident and idle picks the work: every waiting request of the same
// (matrix, op) joins, oldest first, up to k_max vectors, and the group runs as
// multi-vector passes on the slot's stream.  Requests that arrive while others
// run are admitted as soon as a slot frees up, so launches of different
// matrices overlap on the device.  A matrix never has two launches in flight
// (its plan's workspace is shared by its passes).  Each vector's result is what
// the single-vector call computes.
//
// Host-registered matrices become resident through an admission thread: the
// scheduler reserves the matrix's device bytes within the HBM budget (evicting
// idle host-registered matrices, least recently used first, until it fits),
// marks it "admitting" and hands it over; the admission thread copies it to the
// device and plans it on its own stream with no lock held, then publishes the
// plan.  Meanwhile the scheduler keeps dispatching requests on resident
// matrices, and serve_submit / serve_poll / serve_wait proceed.
//
// Request records: a request stays in the table while it is queued, running, or
// finished but not yet reported; the first serve_poll that reports it done, or
// the serve_wait that sees it finish, moves it to a bounded window of recently
// reported requests (so a poll after a wait still answers) and out of the table.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "plan_impl.h"

using Clock = std::chrono::steady_clock;

namespace {

enum Residency { NONRESIDENT = 0, ADMITTING = 1, RESIDENT = 2 };

struct Matrix {
    bool external = false;  // registered plan: caller-owned, never evicted
    spmv_plan_s *plan = nullptr;
    Residency state = NONRESIDENT;
    // host-registered source
    int64_t m = 0, n = 0, nnz = 0;
    int layout = 0, val_t = 0, vec_t = 0;
    const int32_t *h_ptr = nullptr, *h_idx = nullptr;
    const void *h_vals = nullptr;
    void *d_ptr = nullptr, *d_idx = nullptr, *d_vals = nullptr;
    uint64_t footprint = 0;  // device bytes counted against the budget (reserved while admitting)
    uint64_t last_use = 0;
    bool inflight = false;
    int sx = 4;
};

struct Request {
    int mat = 0, op = 0, k = 0;
    const void *in = nullptr;
    void *out = nullptr;
    Clock::time_point submit;
    bool done = false;
    spmv_status status = SPMV_OK;
    double latency_ms = 0.0;
};

struct Reported {  // a request whose completion was reported once
    spmv_status status;
    double latency_ms;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    int mat = -1;
    std::vector<uint64_t> reqs;
};

// Device buffers of an evicted matrix, freed by the admission thread.
struct Garbage {
    spmv_plan_s *plan = nullptr;
    void *d_ptr = nullptr, *d_idx = nullptr, *d_vals = nullptr;
};

int dsize(int t) { return t == SPMV_F64 ? 8 : t == SPMV_F32 ? 4 : 2; }

constexpr size_t REPORTED_WINDOW = 1u << 16;  // recently reported requests kept for serve_poll / serve_wait

}  // namespace

struct serve_s {
    int device = 0;
    uint64_t budget = 0, resident = 0;
    int k_max = 32;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_admit;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    std::unordered_map<uint64_t, Reported> reported;
    std::deque<uint64_t> reported_order;
    std::vector<Matrix> mats;
    std::vector<Slot> slots;
    std::thread sched, admitter;
    cudaStream_t admit_stream = nullptr;
    bool stop = false;
    uint64_t next_id = 1, tick = 0;
    serve_stats_t st{};
    int inflight = 0;
    // admission work handed to the admission thread (under mu)
    std::deque<int> admit_queue;
    std::vector<Garbage> garbage;

    // ---- residency (called with mu held)
    void evict_locked(Matrix &M) {
        garbage.push_back(Garbage{M.plan, M.d_ptr, M.d_idx, M.d_vals});
        M.plan = nullptr;
        M.d_ptr = M.d_idx = M.d_vals = nullptr;
        M.state = NONRESIDENT;
        resident -= M.footprint;
        M.footprint = 0;
        st.evictions++;
        st.resident_matrices--;
    }

    uint64_t estimate(const Matrix &M) const {
        const int64_t major = M.layout == SPMV_CSC_WIDE ? M.n : M.m;
        const int64_t minor = M.layout == SPMV_CSC_WIDE ? M.m : M.n;
        return (uint64_t)M.nnz * (4 + dsize(M.val_t)) + (uint64_t)(major + 1) * 8 +
               std::min<uint64_t>((uint64_t)minor * 32, 232448) * 160 + (4u << 20);
    }

    // Start making matrix `id` resident: reserve its bytes (evicting idle host matrices) and
    // hand it to the admission thread.  False if it cannot start now; *err set if it never can.
    bool start_admission(int id, spmv_status *err) {
        Matrix &M = mats[id];
        *err = SPMV_OK;
        const uint64_t need = estimate(M);
        if (need > budget) {
            *err = SPMV_ERR_BUSY;
            return false;
        }
        while (resident + need > budget) {
            int victim = -1;
            for (int j = 0; j < (int)mats.size(); ++j) {
                Matrix &V = mats[j];
                if (j == id || V.external || V.state != RESIDENT || V.inflight) continue;
                if (victim < 0 || V.last_use < mats[victim].last_use) victim = j;
            }
            if (victim < 0) return false;  // everything resident is busy or admitting: try again later
            evict_locked(mats[victim]);
        }
        M.footprint = need;
        resident += need;
        M.state = ADMITTING;
        admit_queue.push_back(id);
        cv_admit.notify_one();
        return true;
    }

    // ---- the admission thread: frees evicted buffers, copies and plans with no lock held
    void admit_loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            cv_admit.wait(lk, [&] { return stop_admitter || !admit_queue.empty() || !garbage.empty(); });
            std::vector<Garbage> bin;
            bin.swap(garbage);
            int id = -1;
            if (!admit_queue.empty()) {
                id = admit_queue.front();
                admit_queue.pop_front();
            }
            if (id < 0 && bin.empty() && stop_admitter) break;
            // a snapshot of what the copy needs (the record itself may move as mats grows)
            Matrix M = id >= 0 ? mats[id] : Matrix();
            lk.unlock();
            for (auto &g : bin) {
                spmv_plan_destroy(g.plan);
                cudaFree(g.d_ptr);
                cudaFree(g.d_idx);
                cudaFree(g.d_vals);
            }
            spmv_plan_t p = nullptr;
            spmv_status s = SPMV_OK;
            if (id >= 0) s = copy_and_plan(M, &p);
            lk.lock();
            if (id < 0) continue;
            Matrix &R = mats[id];
            resident -= R.footprint;
            if (s == SPMV_OK) {
                R.plan = p;
                R.d_ptr = M.d_ptr;
                R.d_idx = M.d_idx;
                R.d_vals = M.d_vals;
                R.footprint = gbk::plan_footprint(p);
                resident += R.footprint;
                R.state = RESIDENT;
                st.admissions++;
                st.resident_matrices++;
            } else {
                R.footprint = 0;
                R.state = NONRESIDENT;
                // the matrix cannot be made resident: its waiting requests fail
                for (size_t i = 0; i < pending.size();) {
                    if (reqs[pending[i]].mat == id) {
                        finish_locked(pending[i], s);
                        pending.erase(pending.begin() + i);
                    } else {
                        ++i;
                    }
                }
            }
            cv_work.notify_one();
        }
    }
    bool stop_admitter = false;

    // Copy a host matrix to the device and plan it (no lock held); fills M's device pointers.
    spmv_status copy_and_plan(Matrix &M, spmv_plan_t *out) {
        const int64_t major = M.layout == SPMV_CSC_WIDE ? M.n : M.m;
        auto fail = [&](spmv_status s) {
            cudaFree(M.d_ptr);
            cudaFree(M.d_idx);
            cudaFree(M.d_vals);
            M.d_ptr = M.d_idx = M.d_vals = nullptr;
            return s;
        };
        if (cudaMalloc(&M.d_ptr, (size_t)(major + 1) * 4) != cudaSuccess) return fail(SPMV_ERR_OOM);
        if (cudaMalloc(&M.d_idx, std::max<size_t>(16, (size_t)M.nnz * 4)) != cudaSuccess) return fail(SPMV_ERR_OOM);
        if (cudaMalloc(&M.d_vals, std::max<size_t>(16, (size_t)M.nnz * dsize(M.val_t))) != cudaSuccess)
            return fail(SPMV_ERR_OOM);
        cudaStream_t s = admit_stream;
        if (cudaMemcpyAsync(M.d_ptr, M.h_ptr, (size_t)(major + 1) * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            (M.nnz && cudaMemcpyAsync(M.d_idx, M.h_idx, (size_t)M.nnz * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
            (M.nnz && cudaMemcpyAsync(M.d_vals, M.h_vals, (size_t)M.nnz * dsize(M.val_t), cudaMemcpyHostToDevice, s) !=
                          cudaSuccess))
            return fail(SPMV_ERR_CUDA);
        spmv_plan_t p = nullptr;
        spmv_status st_ = spmv_plan(&p, M.m, M.n, M.nnz, M.layout, (const int32_t *)M.d_ptr, (const int32_t *)M.d_idx,
                                    M.d_vals, M.val_t, M.vec_t, s, 0);
        if (st_ != SPMV_OK) return fail(st_);
        *out = p;
        return SPMV_OK;
    }

    // ---- request records (called with mu held)
    void finish_locked(uint64_t rid, spmv_status s) {
        Request &R = reqs[rid];
        R.done = true;
        R.status = s;
        R.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - R.submit).count();
        if (s == SPMV_OK)
            st.completed++;
        else
            st.failed++;
        cv_done.notify_all();
    }

    // The request's completion was reported to the caller: keep it in the bounded window only.
    void retire_locked(uint64_t rid, const Request &R) {
        reported[rid] = Reported{R.status, R.latency_ms};
        reported_order.push_back(rid);
        while (reported_order.size() > REPORTED_WINDOW) {
            reported.erase(reported_order.front());
            reported_order.pop_front();
        }
        reqs.erase(rid);
    }

    // ---- completion and dispatch (called with mu held)
    bool reap() {
        bool any = false;
        for (auto &S : slots) {
            if (!S.busy) continue;
            cudaError_t q = cudaEventQuery(S.ev);
            if (q == cudaErrorNotReady) continue;
            spmv_status status = q == cudaSuccess ? SPMV_OK : SPMV_ERR_CUDA;
            if (q != cudaSuccess) cudaGetLastError();
            for (uint64_t rid : S.reqs) finish_locked(rid, status);
            mats[S.mat].inflight = false;
            S.reqs.clear();
            S.busy = false;
            S.mat = -1;
            inflight--;
            any = true;
        }
        return any;
    }

    bool dispatch() {
        bool any = false;
        for (auto &S : slots) {
            if (S.busy) continue;
            // oldest waiting request whose matrix is resident and idle; non-resident matrices
            // met on the way start their admission (one at a time)
            int pick = -1;
            for (size_t i = 0; i < pending.size(); ++i) {
                const Request &R = reqs[pending[i]];
                Matrix &M = mats[R.mat];
                if (M.state == RESIDENT) {
                    if (M.inflight) continue;
                    pick = (int)i;
                    break;
                }
                if (M.state == NONRESIDENT && admit_queue.empty()) {
                    spmv_status err;
                    if (!start_admission(R.mat, &err) && err != SPMV_OK) {  // can never fit: fail it
                        finish_locked(pending[i], err);
                        pending.erase(pending.begin() + i);
                        --i;
                        any = true;
                    }
                }
            }
            if (pick < 0) break;
            const Request R0 = reqs[pending[pick]];
            Matrix &M = mats[R0.mat];
            std::vector<uint64_t> group;
            int total = 0;
            for (size_t i = pick; i < pending.size();) {
                const Request &R = reqs[pending[i]];
                if (R.mat == R0.mat && R.op == R0.op && (group.empty() || total + R.k <= k_max)) {
                    group.push_back(pending[i]);
                    total += R.k;
                    pending.erase(pending.begin() + i);
                } else {
                    ++i;
                }
            }
            const int64_t len_in = R0.op == SPMV_OP_AX ? M.plan->n : M.plan->m;
            const int64_t len_out = R0.op == SPMV_OP_AX ? M.plan->m : M.plan->n;
            std::vector<const void *> vin;
            std::vector<void *> vout;
            for (uint64_t rid : group) {
                const Request &R = reqs[rid];
                for (int b = 0; b < R.k; ++b) {
                    vin.push_back(static_cast<const char *>(R.in) + (size_t)b * len_in * M.plan->sx);
                    vout.push_back(static_cast<char *>(R.out) + (size_t)b * len_out * M.plan->sx);
                }
            }
            spmv_status s = gbk::run_op(M.plan, R0.op, (int)vin.size(), vin.data(), vout.data(), S.stream);
            if (s != SPMV_OK) {
                for (uint64_t rid : group) finish_locked(rid, s);
                any = true;
                continue;
            }
            cudaEventRecord(S.ev, S.stream);
            S.busy = true;
            S.mat = R0.mat;
            S.reqs = std::move(group);
            M.inflight = true;
            M.last_use = ++tick;
            st.launches++;
            st.vectors += (int64_t)vin.size();
            inflight++;
            st.max_inflight_launches = std::max<int32_t>(st.max_inflight_launches, inflight);
            any = true;
        }
        return any;
    }

    bool admitting() const {
        if (!admit_queue.empty()) return true;
        for (const auto &M : mats)
            if (M.state == ADMITTING) return true;
        return false;
    }

    void loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            const bool a = reap();
            const bool b = dispatch();
            if (stop && pending.empty() && inflight == 0 && !admitting()) break;
            if (!a && !b) {
                if (inflight > 0) {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(20));
                    lk.lock();
                } else {
                    cv_work.wait_for(lk, std::chrono::milliseconds(50));
                }
            }
        }
    }
};

extern "C" {

spmv_status serve_create(serve_t *out, uint64_t hbm_budget_bytes, int32_t k_max, int32_t n_streams) {
    if (!out) return gbk::set_error(SPMV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (k_max < 1 || k_max > 64 || n_streams < 1 || n_streams > 16)
        return gbk::set_error(SPMV_ERR_INVALID_ARG, "k_max must lie in [1, 64] and n_streams in [1, 16]");
    serve_s *s = new (std::nothrow) serve_s();
    if (!s) return gbk::set_error(SPMV_ERR_OOM, "host allocation failed");
    cudaGetDevice(&s->device);
    s->budget = hbm_budget_bytes;
    s->k_max = k_max;
    s->slots.resize(n_streams);
    bool ok = cudaStreamCreateWithFlags(&s->admit_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (auto &S : s->slots) {
        ok = ok && cudaStreamCreateWithFlags(&S.stream, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&S.ev, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        for (auto &T : s->slots) {
            if (T.stream) cudaStreamDestroy(T.stream);
            if (T.ev) cudaEventDestroy(T.ev);
        }
        if (s->admit_stream) cudaStreamDestroy(s->admit_stream);
        delete s;
        return gbk::set_error(SPMV_ERR_CUDA, "stream/event creation failed");
    }
    s->sched = std::thread([s] { s->loop(); });
    s->admitter = std::thread([s] { s->admit_loop(); });
    *out = s;
    return SPMV_OK;
}

spmv_status serve_register(serve_t s, spmv_plan_t plan, int32_t *mat_id) {
    if (!s || !plan || !mat_id) return gbk::set_error(SPMV_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t fp = gbk::plan_footprint(plan);
    if (s->resident + fp > s->budget) return gbk::set_error(SPMV_ERR_BUSY, "plan does not fit the HBM budget");
    Matrix M;
    M.external = true;
    M.plan = plan;
    M.state = RESIDENT;
    M.m = plan->m;
    M.n = plan->n;
    M.nnz = plan->nnz;
    M.layout = plan->layout;
    M.val_t = plan->val_t;
    M.vec_t = plan->vec_t;
    M.sx = plan->sx;
    M.footprint = fp;
    s->resident += fp;
    s->st.resident_matrices++;
    s->mats.push_back(M);
    *mat_id = (int32_t)s->mats.size() - 1;
    return SPMV_OK;
}

spmv_status serve_register_host(serve_t s, int64_t m, int64_t n, int64_t nnz, int32_t layout, const int32_t *ptr,
                                const int32_t *idx, const void *vals, int32_t val_dtype, int32_t vec_dtype,
                                int32_t *mat_id) {
    if (!s || !ptr || !mat_id || (nnz > 0 && (!idx || !vals)))
        return gbk::set_error(SPMV_ERR_INVALID_ARG, "null argument");
    if (layout != SPMV_CSC_WIDE && layout != SPMV_CSR_TALL) return gbk::set_error(SPMV_ERR_INVALID_ARG, "bad layout");
    if (m < 0 || n < 0 || nnz < 0) return gbk::set_error(SPMV_ERR_INVALID_ARG, "negative size");
    std::lock_guard<std::mutex> lk(s->mu);
    Matrix M;
    M.m = m;
    M.n = n;
    M.nnz = nnz;
    M.layout = layout;
    M.val_t = val_dtype;
    M.vec_t = vec_dtype;
    M.sx = dsize(vec_dtype);
    M.h_ptr = ptr;
    M.h_idx = idx;
    M.h_vals = vals;
    s->mats.push_back(M);
    *mat_id = (int32_t)s->mats.size() - 1;
    return SPMV_OK;
}

spmv_status serve_submit(serve_t s, int32_t mat_id, int32_t op, int32_t k, const void *in, void *out,
                         uint64_t *req_id) {
    if (!s || !req_id || !in || !out) return gbk::set_error(SPMV_ERR_INVALID_ARG, "null argument");
    if (op != SPMV_OP_AX && op != SPMV_OP_VTA) return gbk::set_error(SPMV_ERR_INVALID_ARG, "bad op");
    if (k < 1 || k > 4096) return gbk::set_error(SPMV_ERR_INVALID_ARG, "k must lie in [1, 4096]");
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return gbk::set_error(SPMV_ERR_INVALID_ARG, "vectors must be 16-byte aligned device memory");
    std::lock_guard<std::mutex> lk(s->mu);
    if (mat_id < 0 || mat_id >= (int)s->mats.size()) return gbk::set_error(SPMV_ERR_NOT_FOUND, "unknown matrix");
    const Matrix &M = s->mats[mat_id];
    const int64_t len_in = op == SPMV_OP_AX ? M.n : M.m;
    const int64_t len_out = op == SPMV_OP_AX ? M.m : M.n;
    if (k > 1 && (((size_t)len_in * M.sx) % 16 || ((size_t)len_out * M.sx) % 16))
        return gbk::set_error(SPMV_ERR_INVALID_ARG, "with k > 1 every vector must start on a 16-byte boundary");
    const uint64_t id = s->next_id++;
    Request R;
    R.mat = mat_id;
    R.op = op;
    R.k = k;
    R.in = in;
    R.out = out;
    R.submit = Clock::now();
    s->reqs.emplace(id, R);
    s->pending.push_back(id);
    s->st.submitted++;
    *req_id = id;
    s->cv_work.notify_one();
    return SPMV_OK;
}

spmv_status serve_poll(serve_t s, uint64_t req_id, int32_t *done, double *latency_ms) {
    if (!s || !done) return gbk::set_error(SPMV_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) {
        auto r = s->reported.find(req_id);
        if (r == s->reported.end()) return gbk::set_error(SPMV_ERR_NOT_FOUND, "unknown request");
        *done = 1;
        if (latency_ms) *latency_ms = r->second.latency_ms;
        if (r->second.status != SPMV_OK) return gbk::set_error(r->second.status, "request failed");
        return SPMV_OK;
    }
    const Request R = it->second;
    *done = R.done ? 1 : 0;
    if (latency_ms) *latency_ms = R.latency_ms;
    if (R.done) s->retire_locked(req_id, R);
    if (R.done && R.status != SPMV_OK) return gbk::set_error(R.status, "request failed");
    return SPMV_OK;
}

spmv_status serve_wait(serve_t s, uint64_t req_id, int32_t timeout_ms) {
    if (!s) return gbk::set_error(SPMV_ERR_INVALID_ARG, "null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->reqs.find(req_id) == s->reqs.end()) {
        auto r = s->reported.find(req_id);
        if (r == s->reported.end()) return gbk::set_error(SPMV_ERR_NOT_FOUND, "unknown request");
        if (r->second.status != SPMV_OK) return gbk::set_error(r->second.status, "request failed");
        return SPMV_OK;
    }
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)), [&] {
        auto it = s->reqs.find(req_id);
        return it == s->reqs.end() || it->second.done;  // gone: another waiter reported it
    });
    if (!ok) return gbk::set_error(SPMV_ERR_TIMEOUT, "request not finished within the timeout");
    spmv_status st;
    auto it = s->reqs.find(req_id);
    if (it != s->reqs.end()) {
        const Request R = it->second;
        st = R.status;
        s->retire_locked(req_id, R);
    } else {
        auto r = s->reported.find(req_id);
        st = r == s->reported.end() ? SPMV_OK : r->second.status;
    }
    if (st != SPMV_OK) return gbk::set_error(st, "request failed");
    return SPMV_OK;
}

spmv_status serve_stats(serve_t s, serve_stats_t *out) {
    if (!s || !out) return gbk::set_error(SPMV_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->resident_bytes = s->resident;
    out->tracked_requests = (int64_t)s->reqs.size();
    return SPMV_OK;
}

spmv_status serve_destroy(serve_t s) {
    if (!s) return SPMV_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->sched.joinable()) s->sched.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto &M : s->mats)
            if (!M.external && M.state == RESIDENT) s->evict_locked(M);
        s->stop_admitter = true;
    }
    s->cv_admit.notify_all();
    if (s->admitter.joinable()) s->admitter.join();
    for (auto &S : s->slots) {
        cudaStreamDestroy(S.stream);
        cudaEventDestroy(S.ev);
    }
    cudaStreamDestroy(s->admit_stream);
    delete s;
    return SPMV_OK;
}

}  // extern "C"
