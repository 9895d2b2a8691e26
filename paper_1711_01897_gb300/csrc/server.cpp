// Request server: admission by HBM budget in arrival order, one worker thread
// and CUDA stream per slot, host-side tree construction overlapping other
// requests' device work.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "bem_host_internal.h"

using namespace bem;

namespace {

double steady_ms()
{
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Req {
    int64_t id = 0;
    std::vector<double> V;
    std::vector<int32_t> T;
    std::vector<double> x, y;  // complex as interleaved pairs
    int32_t op = 0, prec = 0, leaf = 32;
    double k = 0, eps = 1e-4, eta = 1.2, dry_ms = 0;
    int state = BEM_REQ_QUEUED;
    int status = BEM_OK;
    double t_submit = 0, t_admit = 0, t_done = 0, asm_ms = 0;
    int64_t reserved = 0, integrals = 0;
};

}  // namespace

struct bem_server_s {
    int64_t budget = 0;
    int slots = 0;
    int flags = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_budget, cv_done;
    std::deque<int64_t> queue;           // submitted, not yet taken by a worker
    std::deque<int64_t> waiting;         // prepared, waiting for budget, arrival order
    std::map<int64_t, std::unique_ptr<Req>> reqs;
    int64_t next_id = 1;
    int64_t in_use = 0, peak = 0;
    int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, running = 0;
    bool stopping = false;
    std::vector<std::thread> workers;

    void worker();
    void finish(Req *r, int status, int64_t bytes);
};

void bem_server_s::finish(Req *r, int status, int64_t bytes)
{
    std::lock_guard<std::mutex> lk(mu);
    in_use -= bytes;
    if (r->state == BEM_REQ_RUNNING) --running;
    r->status = status;
    r->state = status == BEM_OK ? BEM_REQ_DONE : BEM_REQ_FAILED;
    r->t_done = steady_ms();
    if (status == BEM_OK) ++completed;
    else ++failed;
    cv_budget.notify_all();
    cv_done.notify_all();
}

void bem_server_s::worker()
{
    const bool dry = flags & BEM_SERVER_DRY_RUN;
    cudaStream_t st = nullptr;
    if (!dry) {
        cudaSetDevice(device);
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    }
    for (;;) {
        Req *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stopping || !queue.empty(); });
            if (queue.empty()) break;
            r = reqs[queue.front()].get();
            queue.pop_front();
            r->state = BEM_REQ_PREPARING;
        }
        const int64_t nt = (int64_t)r->T.size() / 3, nv = (int64_t)r->V.size() / 3;
        // host part: validation, adjacency, trees; exact device bytes
        bem_mesh M = nullptr;
        bem_hmat H = nullptr;
        int64_t bytes = 0;
        int rc = BEM_OK;
        if (dry) {
            bytes = nt * 1024;
        } else {
            rc = mesh_create_impl(r->V.data(), nv, r->T.data(), nt, kHostOnly, &M);
            if (rc == BEM_OK) rc = hmat_build_tree_impl(M, r->leaf, r->eta, kHostOnly, &H);
            if (rc == BEM_OK) bytes = hmat_device_bytes(H, r->k != 0.0);
        }
        if (rc == BEM_OK && bytes > budget) rc = BEM_E_OOM;
        if (rc != BEM_OK) {
            if (H) hmat_free_synced(H);
            if (M) mesh_free_synced(M);
            finish(r, rc, 0);
            continue;
        }
        // admission: in arrival order, when the bytes fit next to the running ones
        {
            std::unique_lock<std::mutex> lk(mu);
            waiting.push_back(r->id);
            std::sort(waiting.begin(), waiting.end());
            cv_budget.wait(lk, [&] {
                return waiting.front() == r->id && in_use + bytes <= budget;
            });
            waiting.pop_front();
            in_use += bytes;
            peak = std::max(peak, in_use);
            r->reserved = bytes;
            r->state = BEM_REQ_RUNNING;
            r->t_admit = steady_ms();
            ++running;
            cv_budget.notify_all();
        }
        // device part on this worker's stream
        if (dry) {
            std::this_thread::sleep_for(std::chrono::duration<double, std::milli>(r->dry_ms));
            r->y = r->x;
            finish(r, BEM_OK, bytes);
            continue;
        }
        if (!st) rc = BEM_E_CUDA;
        if (rc == BEM_OK) rc = mesh_upload(M, st);
        if (rc == BEM_OK) rc = hmat_upload(H, st);
        if (rc == BEM_OK) rc = hmat_assemble(H, r->op, r->k, r->eps, r->prec, st);
        if (rc == BEM_OK) {
            r->y.assign(r->x.size(), 0.0);
            rc = hmat_matvec(H, r->x.data(), r->y.data(), 1, st);
        }
        if (rc == BEM_OK) {
            bem_hmat_stats s;
            if (hmat_stats(H, &s) == BEM_OK) {
                r->integrals = s.near_entries + s.far_entries;
                r->asm_ms = s.time_near_ms + s.time_far_ms;
            }
        }
        cudaStreamSynchronize(st);
        if (H) hmat_free_synced(H);
        if (M) mesh_free_synced(M);
        cudaStreamSynchronize(st);  // stream-ordered frees complete before the bytes return
        finish(r, rc, bytes);
    }
    if (st) cudaStreamDestroy(st);
}

extern "C" {

int bem_server_create(int64_t hbm_budget_bytes, int32_t max_slots, int32_t flags, bem_server *out)
{
    if (!out) return BEM_E_ARG;
    *out = nullptr;
    if (hbm_budget_bytes <= 0 || max_slots < 1 || max_slots > 64) {
        set_last_error("bad server arguments");
        return BEM_E_ARG;
    }
    auto S = std::make_unique<bem_server_s>();
    S->budget = hbm_budget_bytes;
    S->slots = max_slots;
    S->flags = flags;
    if (!(flags & BEM_SERVER_DRY_RUN)) {
        if (cudaGetDevice(&S->device) != cudaSuccess) {
            set_last_error("no CUDA device");
            return BEM_E_CUDA;
        }
    }
    for (int i = 0; i < max_slots; ++i) S->workers.emplace_back([s = S.get()] { s->worker(); });
    *out = S.release();
    return BEM_OK;
}

int bem_server_submit(bem_server S, const bem_request *q, int64_t *req_id)
{
    if (!S || !q || !req_id) return BEM_E_ARG;
    if (!q->vertices || !q->triangles || !q->x || q->n_vertices < 3 || q->n_triangles < 1 ||
        q->op < 0 || q->op > 2 || (q->prec != BEM_FP64 && q->prec != BEM_MIXED) ||
        !(q->aca_eps > 0) || q->leaf_size < 1 || !(q->eta > 0)) {
        set_last_error("bad request");
        return BEM_E_ARG;
    }
    auto r = std::make_unique<Req>();
    r->V.assign(q->vertices, q->vertices + 3 * q->n_vertices);
    r->T.assign(q->triangles, q->triangles + 3 * q->n_triangles);
    const int64_t nx = q->n_triangles * (q->k != 0.0 ? 2 : 1);
    const double *x = static_cast<const double *>(q->x);
    r->x.assign(x, x + nx);
    r->op = q->op;
    r->prec = q->prec;
    r->leaf = q->leaf_size;
    r->k = q->k;
    r->eps = q->aca_eps;
    r->eta = q->eta;
    r->dry_ms = q->dry_run_ms > 0 ? q->dry_run_ms : 0.0;
    r->t_submit = steady_ms();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return BEM_E_STATE;
    r->id = S->next_id++;
    *req_id = r->id;
    S->queue.push_back(r->id);
    S->reqs[r->id] = std::move(r);
    ++S->submitted;
    S->cv_work.notify_one();
    return BEM_OK;
}

static void fill_info(const Req &r, bem_request_info *info)
{
    if (!info) return;
    info->state = r.state;
    info->status = r.status;
    info->t_submit_ms = r.t_submit;
    info->t_admit_ms = r.t_admit;
    info->t_done_ms = r.t_done;
    info->reserved_bytes = r.reserved;
    info->integrals = r.integrals;
    info->assembly_ms = r.asm_ms;
}

int bem_server_poll(bem_server S, int64_t id, bem_request_info *info)
{
    if (!S) return BEM_E_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return BEM_E_ARG;
    fill_info(*it->second, info);
    return BEM_OK;
}

int bem_server_wait(bem_server S, int64_t id, int64_t timeout_ms, bem_request_info *info, void *y)
{
    if (!S) return BEM_E_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return BEM_E_ARG;
    Req *r = it->second.get();
    auto done = [&] {
        return r->state == BEM_REQ_DONE || r->state == BEM_REQ_FAILED ||
               r->state == BEM_REQ_CANCELLED;
    };
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, done);
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        fill_info(*r, info);
        set_last_error("request not finished within the timeout");
        return BEM_E_TIMEOUT;
    }
    fill_info(*r, info);
    int status = r->status;
    if (r->state == BEM_REQ_DONE && y) std::memcpy(y, r->y.data(), r->y.size() * sizeof(double));
    S->reqs.erase(it);
    return status;
}

int bem_server_cancel(bem_server S, int64_t id)
{
    if (!S) return BEM_E_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return BEM_E_ARG;
    auto q = std::find(S->queue.begin(), S->queue.end(), id);
    if (q == S->queue.end()) return BEM_E_STATE;
    S->queue.erase(q);
    it->second->state = BEM_REQ_CANCELLED;
    it->second->status = BEM_E_STATE;
    ++S->cancelled;
    S->cv_done.notify_all();
    return BEM_OK;
}

int bem_server_stats_get(bem_server S, bem_server_stats *out)
{
    if (!S || !out) return BEM_E_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->failed = S->failed;
    out->cancelled = S->cancelled;
    out->queued = (int64_t)S->queue.size() + (int64_t)S->waiting.size();
    out->running = S->running;
    out->reserved_bytes = S->in_use;
    out->peak_reserved_bytes = S->peak;
    out->budget_bytes = S->budget;
    return BEM_OK;
}

int bem_server_destroy(bem_server S)
{
    if (!S) return BEM_E_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        for (int64_t id : S->queue) {
            S->reqs[id]->state = BEM_REQ_CANCELLED;
            S->reqs[id]->status = BEM_E_STATE;
            ++S->cancelled;
        }
        S->queue.clear();
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
    for (auto &t : S->workers) t.join();
    delete S;
    return BEM_OK;
}

}  // extern "C"
