// Request server with continuous batching.
//
// Worker threads do each request's host part (mesh validation, adjacency,
// cluster and block trees, exact device bytes).  One engine thread admits
// prepared requests in arrival order while their bytes fit the HBM budget
// (evicting idle resident H-matrices, least recently used first), and puts
// every request admitted since its last launch into one batch on a free
// engine stream: uploads, each request's near field, then ONE persistent ACA
// launch per kind of matrix (operator, number type, precision) over the
// admissible blocks of all the batch's requests, then the products.  While a
// batch runs, requests that arrive are admitted into the next batch, which
// can start on the other stream.  Assembled H-matrices stay resident (their
// bytes stay reserved) until the budget needs them, so a later request that
// names an earlier one (bem_request.reuse) only runs the product.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
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

constexpr int kEngineStreams = 2;   // batches in flight at once
constexpr int kBatchMax = 64;       // requests per batch
// A free stream waits up to this long after the oldest admitted request for
// requests still being prepared, so that they share the launch.
constexpr double kBatchWindowMs = 2.0;
// Requests with at least this many triangles are large: they are batched
// apart from the small ones, at most one large batch runs at a time, and its
// ACA launch leaves a quarter of the SMs to the small batches on the other
// stream (so that a large assembly does not hold up small requests).
constexpr int64_t kLargeTriangles = 40000;
constexpr double kLargeSmShare = 0.75;
constexpr double kLargeWaitMs = 50.0;
// Admission: a request that does not fit the budget lets younger ones pass;
// after this long its bytes are held for it.  At most kMaxLargeRunning large
// requests run at once.
constexpr double kBypassMs = 300.0;
constexpr int64_t kMaxLargeRunning = 2;
// Large requests may hold at most this share of the budget (running and
// admitted), so that small requests always find room.
constexpr double kLargeBudgetShare = 0.7;

// An assembled H-matrix kept on the device after its request finished.
struct Resident {
    int64_t id = 0;          // the request that assembled it
    bem_mesh M = nullptr;
    bem_hmat H = nullptr;
    int64_t bytes = 0;
    int32_t op = 0, prec = 0;
    double k = 0, eps = 0;
    int64_t nt = 0;
    double last_use = 0;
    int users = 0;           // admitted requests that apply it
};

struct Req {
    int64_t id = 0;
    std::vector<double> V;
    std::vector<int32_t> T;
    std::vector<double> x, y;  // complex as interleaved pairs
    int32_t op = 0, prec = 0, leaf = 32;
    double k = 0, eps = 1e-4, eta = 1.2, dry_ms = 0;
    int64_t reuse = 0;         // request whose resident matrix to apply (0: assemble)
    int state = BEM_REQ_QUEUED;
    int status = BEM_OK;
    double t_submit = 0, t_admit = 0, t_done = 0, asm_ms = 0, t_ready = 0, t_launch = 0;
    int64_t reserved = 0, integrals = 0;
    int32_t launch_reqs = 0;   // requests that shared its ACA launch
    int32_t reused = 0;        // 1: applied a resident matrix, no assembly
    // host objects between preparation and completion
    bem_mesh M = nullptr;
    bem_hmat H = nullptr;
    int64_t bytes = 0;
    Resident *res = nullptr;   // the resident matrix a product-only request applies
};

struct Batch {
    int slot = -1;
    bool large = false;
    std::vector<Req *> reqs;
    double t_launch = 0;
};

bool is_large(const Req *r)
{
    return r->res == nullptr && (int64_t)r->T.size() / 3 >= kLargeTriangles;
}

}  // namespace

struct bem_server_s {
    int64_t budget = 0;
    int slots = 0;
    int flags = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_engine, cv_done;
    std::deque<int64_t> queue;           // submitted, not yet taken by a worker
    std::deque<int64_t> prepared;        // host part done, waiting for admission
    std::vector<Req *> admitted;         // admitted, not yet in a batch
    std::map<int64_t, std::unique_ptr<Req>> reqs;
    std::list<Resident> residents;
    int64_t next_id = 1;
    int64_t in_use = 0, peak = 0;
    int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, running = 0;
    int64_t running_large = 0, in_use_large = 0;
    int64_t evictions = 0, reuse_hits = 0, fused_launches = 0, fused_requests = 0;
    int64_t max_launch_requests = 0;
    int preparing = 0;
    bool stopping = false;
    std::vector<std::thread> workers;
    std::thread engine;
    cudaStream_t streams[kEngineStreams] = {};
    cudaEvent_t events[kEngineStreams] = {};
    void *staging[kEngineStreams] = {};     // page-locked work-list staging per stream
    size_t staging_bytes[kEngineStreams] = {};
    Batch inflight[kEngineStreams];

    void worker();
    void engine_loop();
    bool evict_one();
    void launch(Batch &b);
    void complete(Batch &b);
    void finish_locked(Req *r, int status);
    Resident *find_resident(int64_t id);
};

Resident *bem_server_s::find_resident(int64_t id)
{
    for (Resident &R : residents)
        if (R.id == id) return &R;
    return nullptr;
}

// Frees the least recently used idle resident matrix; false if none.
// Called with mu held.
bool bem_server_s::evict_one()
{
    auto victim = residents.end();
    for (auto it = residents.begin(); it != residents.end(); ++it)
        if (it->users == 0 && (victim == residents.end() || it->last_use < victim->last_use))
            victim = it;
    if (victim == residents.end()) return false;
    if (victim->H) hmat_free_synced(victim->H);
    if (victim->M) mesh_free_synced(victim->M);
    in_use -= victim->bytes;
    ++evictions;
    residents.erase(victim);
    return true;
}

// Called with mu held.
void bem_server_s::finish_locked(Req *r, int status)
{
    if (r->state == BEM_REQ_RUNNING) {
        --running;
        if (is_large(r)) {
            --running_large;
            in_use_large -= r->bytes;
        }
    }
    r->status = status;
    r->state = status == BEM_OK ? BEM_REQ_DONE : BEM_REQ_FAILED;
    r->t_done = steady_ms();
    if (status == BEM_OK) ++completed;
    else ++failed;
    cv_done.notify_all();
    cv_engine.notify_all();
}

void bem_server_s::worker()
{
    const bool dry = flags & BEM_SERVER_DRY_RUN;
    for (;;) {
        Req *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stopping || !queue.empty(); });
            if (queue.empty()) break;
            r = reqs[queue.front()].get();
            queue.pop_front();
            r->state = BEM_REQ_PREPARING;
            ++preparing;
        }
        int rc = BEM_OK;
        if (r->reuse > 0) {
            // a product with an earlier request's matrix: nothing to build
            // while it is resident (checked again at admission)
            r->bytes = 0;
        } else if (dry) {
            r->bytes = (int64_t)r->T.size() / 3 * 1024;
        } else {
            const int64_t nt = (int64_t)r->T.size() / 3, nv = (int64_t)r->V.size() / 3;
            cudaSetDevice(device);
            rc = mesh_create_impl(r->V.data(), nv, r->T.data(), nt, kHostOnly, &r->M);
            if (rc == BEM_OK) rc = hmat_build_tree_impl(r->M, r->leaf, r->eta, kHostOnly, &r->H);
            if (rc == BEM_OK) r->bytes = hmat_device_bytes(r->H, r->k != 0.0);
        }
        if (rc == BEM_OK && r->bytes > budget) rc = BEM_E_OOM;
        std::lock_guard<std::mutex> lk(mu);
        --preparing;
        if (rc != BEM_OK || r->state == BEM_REQ_CANCELLED) {
            if (r->H) hmat_free_synced(r->H);
            if (r->M) mesh_free_synced(r->M);
            r->H = nullptr;
            r->M = nullptr;
            if (r->state != BEM_REQ_CANCELLED) finish_locked(r, rc);
            continue;
        }
        r->t_ready = steady_ms();
        prepared.push_back(r->id);
        std::sort(prepared.begin(), prepared.end());
        cv_engine.notify_all();
    }
}

// Device work of one batch on its engine stream (mu not held).  Requests
// that fail here are finished at once; the rest complete in complete().
void bem_server_s::launch(Batch &b)
{
    const bool dry = flags & BEM_SERVER_DRY_RUN;
    cudaStream_t st = streams[b.slot];
    b.t_launch = steady_ms();
    for (Req *r : b.reqs) r->t_launch = b.t_launch;
    if (dry) {
        // one simulated ACA launch per kind of matrix among the assemblies
        std::map<std::tuple<int, int, int>, int> kinds;
        for (Req *r : b.reqs)
            if (!r->res) ++kinds[{r->op, r->k != 0.0, r->prec}];
        std::lock_guard<std::mutex> lk(mu);
        for (Req *r : b.reqs)
            if (!r->res) r->launch_reqs = kinds[{r->op, r->k != 0.0, r->prec}];
        for (auto &kv : kinds) {
            ++fused_launches;
            fused_requests += kv.second;
            max_launch_requests = std::max(max_launch_requests, (int64_t)kv.second);
        }
        return;
    }
    cudaSetDevice(device);
    std::vector<Req *> ok;
    for (Req *r : b.reqs) {
        if (r->res) {        // product only: nothing to assemble
            ok.push_back(r);
            continue;
        }
        int rc = mesh_upload(r->M, st);
        if (rc == BEM_OK) rc = hmat_upload(r->H, st);
        if (rc == BEM_OK) rc = guarded_call([&]() -> int {
            int c = assemble_begin(r->H, r->op, r->k, r->eps, r->prec, st);
            if (c != BEM_OK) return c;
            assemble_pool(r->H, st);
            enqueue_near(r->H, st, false);
            return BEM_OK;
        });
        if (rc != BEM_OK) {
            r->status = rc;
            continue;
        }
        ok.push_back(r);
    }
    // one ACA launch per kind of matrix over all the batch's blocks
    std::map<std::tuple<int, int, int, int>, std::vector<Req *>> kinds;
    for (Req *r : ok)
        if (!r->res) kinds[{r->op, r->k != 0.0, r->prec, hmat_has_rules(r->H) ? 1 : 0}].push_back(r);
    // each launch's work list goes through its own region of this stream's
    // page-locked staging (the copies run later on the stream, so no region
    // is reused within a batch); the staging grows (rarely) while the
    // stream has no work queued
    std::vector<size_t> bound;
    size_t total = 0;
    for (auto &kv : kinds) {
        size_t need = kv.second.size() * sizeof(AcaJob) + 256 + 4096;
        for (Req *r : kv.second) need += (size_t)(r->T.size() / 3) * 4 * sizeof(int64_t);
        need = (need + 255) / 256 * 256;
        bound.push_back(need);
        total += need;
    }
    if (staging_bytes[b.slot] < total) {
        void *p = nullptr;
        const size_t want = std::max<size_t>(total, size_t(32) << 20);
        if (cudaHostAlloc(&p, want, cudaHostAllocDefault) == cudaSuccess) {
            if (staging[b.slot]) cudaFreeHost(staging[b.slot]);
            staging[b.slot] = p;
            staging_bytes[b.slot] = want;
        } else {
            cudaGetLastError();
        }
    }
    const bool staged = staging[b.slot] && staging_bytes[b.slot] >= total;
    size_t at = 0, q = 0;
    for (auto &kv : kinds) {
        std::vector<bem_hmat> hs;
        for (Req *r : kv.second) hs.push_back(r->H);
        void *region = staged ? (char *)staging[b.slot] + at : nullptr;
        const size_t region_bytes = staged ? bound[q] : 0;
        at += bound[q++];
        int rc = guarded_call([&]() -> int {
            return enqueue_aca_fused(hs, st, b.large ? kLargeSmShare : 1.0, region, region_bytes);
        });
        for (Req *r : kv.second) {
            r->launch_reqs = (int32_t)kv.second.size();
            if (rc != BEM_OK) r->status = rc;
        }
        if (rc == BEM_OK) {
            std::lock_guard<std::mutex> lk(mu);
            ++fused_launches;
            fused_requests += (int64_t)kv.second.size();
            max_launch_requests = std::max(max_launch_requests, (int64_t)kv.second.size());
        }
    }
    for (Req *r : ok)
        if (!r->res && r->status == BEM_OK)
            r->status = guarded_call([&]() -> int {
                enqueue_finish(r->H, st, false);
                return BEM_OK;
            });
    cudaEventRecord(events[b.slot], st);
}

// After the batch's event: pool overflows are redone alone, then the
// products; every request is finished and its matrix kept resident.
void bem_server_s::complete(Batch &b)
{
    const bool dry = flags & BEM_SERVER_DRY_RUN;
    cudaStream_t st = streams[b.slot];
    if (dry) {
        double longest = 0;
        for (Req *r : b.reqs) longest = std::max(longest, r->dry_ms);
        const double wait = b.t_launch + longest - steady_ms();
        if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double, std::milli>(wait));
    } else {
        cudaSetDevice(device);
        cudaStreamSynchronize(st);
    }
    for (Req *r : b.reqs) {
        int rc = r->status;
        bem_hmat H = r->res ? r->res->H : r->H;
        if (dry) {
            r->y = r->x;
        } else {
            if (rc == BEM_OK && !r->res) {
                if (assemble_overflowed(H))
                    rc = hmat_assemble(H, r->op, r->k, r->eps, r->prec, st);
                else
                    rc = guarded_call([&]() -> int {
                        assemble_end(H, st);
                        return BEM_OK;
                    });
            }
            if (rc == BEM_OK) {
                r->y.assign(r->x.size(), 0.0);
                rc = hmat_matvec(H, r->x.data(), r->y.data(), 1, st);
            }
            if (rc == BEM_OK && !r->res) {
                bem_hmat_stats s;
                if (hmat_stats(H, &s) == BEM_OK) {
                    r->integrals = s.near_entries + s.far_entries;
                    r->asm_ms = s.time_near_ms + s.time_far_ms;
                }
            }
        }
        std::lock_guard<std::mutex> lk(mu);
        if (r->res) {
            --r->res->users;
            r->res->last_use = steady_ms();
        } else if (rc == BEM_OK) {
            Resident R;
            R.id = r->id;
            R.M = r->M;
            R.H = r->H;
            R.bytes = r->bytes;
            R.op = r->op;
            R.prec = r->prec;
            R.k = r->k;
            R.eps = r->eps;
            R.nt = (int64_t)r->T.size() / 3;
            R.last_use = steady_ms();
            residents.push_back(R);
        } else {
            if (r->H) hmat_free_synced(r->H);
            if (r->M) mesh_free_synced(r->M);
            in_use -= r->bytes;
        }
        r->H = nullptr;
        r->M = nullptr;
        r->res = nullptr;
        finish_locked(r, rc);
    }
    b.reqs.clear();
}

void bem_server_s::engine_loop()
{
    const bool dry = flags & BEM_SERVER_DRY_RUN;
    if (!dry) cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool any_inflight = false;
        for (auto &b : inflight) any_inflight |= !b.reqs.empty();
        // finished batches
        for (int s = 0; s < kEngineStreams; ++s) {
            Batch &b = inflight[s];
            if (b.reqs.empty()) continue;
            bool done;
            if (dry) {
                double longest = 0;
                for (Req *r : b.reqs) longest = std::max(longest, r->dry_ms);
                done = steady_ms() >= b.t_launch + longest;
            } else {
                done = cudaEventQuery(events[s]) != cudaErrorNotReady;
            }
            if (done) {
                lk.unlock();
                complete(b);
                lk.lock();
            }
        }
        // admission in arrival order, evicting idle resident matrices.  A
        // request that does not fit the budget lets younger ones pass; once it
        // has waited kBypassMs its bytes are held for it, so that the younger
        // ones only use what is left and it starts as soon as running requests
        // give back enough.
        int64_t held[2] = {0, 0};   // bytes held for waiting small / large requests
        for (size_t qi = 0; qi < prepared.size();) {
            if (running >= slots) break;
            Req *r = reqs[prepared[qi]].get();
            const bool lg = is_large(r);
            if (lg && running_large >= kMaxLargeRunning) {
                ++qi;
                continue;
            }
            if (r->reuse > 0) {
                Resident *R = find_resident(r->reuse);
                if (!R) {
                    auto src = reqs.find(r->reuse);
                    if (src != reqs.end() && src->second->state != BEM_REQ_DONE &&
                        src->second->state != BEM_REQ_FAILED &&
                        src->second->state != BEM_REQ_CANCELLED) {
                        ++qi;   // its assembly is still on the way: wait for it
                        continue;
                    }
                    // failed, cancelled or evicted
                    prepared.erase(prepared.begin() + qi);
                    set_last_error("the request to reuse has no resident matrix");
                    r->state = BEM_REQ_RUNNING;
                    ++running;
                    finish_locked(r, BEM_E_STATE);
                    continue;
                }
                if ((int64_t)r->x.size() != R->nt * (R->k != 0.0 ? 2 : 1)) {
                    prepared.erase(prepared.begin() + qi);
                    set_last_error("vector length does not match the resident matrix");
                    r->state = BEM_REQ_RUNNING;
                    ++running;
                    finish_locked(r, BEM_E_ARG);
                    continue;
                }
                r->res = R;
                r->op = R->op;
                r->k = R->k;
                r->eps = R->eps;
                r->prec = R->prec;
                r->reused = 1;
                ++R->users;
                ++reuse_hits;
            } else {
                const int64_t h = held[lg ? 1 : 0];
                // (a large request alone may exceed the share: it then runs by itself)
                const bool large_room =
                    !lg || in_use_large == 0 ||
                    (double)(in_use_large + r->bytes + h) <= kLargeBudgetShare * (double)budget;
                while (large_room && in_use + r->bytes + h > budget && evict_one()) {
                }
                if (!large_room || in_use + r->bytes + h > budget) {
                    if (steady_ms() - r->t_ready >= kBypassMs) held[lg ? 1 : 0] += r->bytes;
                    ++qi;
                    continue;
                }
                in_use += r->bytes;
                if (lg) in_use_large += r->bytes;
                peak = std::max(peak, in_use);
            }
            prepared.erase(prepared.begin() + qi);
            r->reserved = r->bytes;
            r->state = BEM_REQ_RUNNING;
            r->t_admit = steady_ms();
            ++running;
            if (lg) ++running_large;
            admitted.push_back(r);
        }
        // a batch of everything admitted, on a free stream
        int free_slot = -1;
        for (int s = 0; s < kEngineStreams; ++s)
            if (inflight[s].reqs.empty()) {
                free_slot = s;
                break;
            }
        const bool more_coming = preparing > 0 || !queue.empty() || !prepared.empty();
        const bool window_over =
            !admitted.empty() && steady_ms() - admitted.front()->t_admit >= kBatchWindowMs;
        bool large_inflight = false;
        for (auto &b : inflight) large_inflight |= !b.reqs.empty() && b.large;
        if (!admitted.empty() && free_slot >= 0 &&
            (!more_coming || window_over || admitted.size() >= (size_t)kBatchMax ||
             running >= slots)) {
            // a batch of one size class: the small requests, else (if no large
            // batch is running) the large ones
            bool any_small = false, any_large = false;
            for (Req *r : admitted) (is_large(r) ? any_large : any_small) = true;
            // small first, unless the oldest admitted request is a large one
            // that has waited long enough (no starvation under a stream of
            // small requests)
            const bool large_overdue = is_large(admitted.front()) &&
                                       steady_ms() - admitted.front()->t_admit > kLargeWaitMs;
            const bool take_large = !any_small || (large_overdue && !large_inflight);
            if (!take_large || !large_inflight) {
                Batch &b = inflight[free_slot];
                b.slot = free_slot;
                b.large = take_large;
                b.reqs.clear();
                for (auto it = admitted.begin();
                     it != admitted.end() && b.reqs.size() < (size_t)kBatchMax;) {
                    if (is_large(*it) == take_large) {
                        b.reqs.push_back(*it);
                        it = admitted.erase(it);
                    } else {
                        ++it;
                    }
                }
                lk.unlock();
                launch(b);
                lk.lock();
                continue;
            }
        }
        any_inflight = false;
        for (auto &b : inflight) any_inflight |= !b.reqs.empty();
        if (stopping && !any_inflight && admitted.empty() && preparing == 0 && queue.empty() &&
            prepared.empty())
            break;
        if (stopping && !any_inflight && admitted.empty() && preparing == 0 && queue.empty()) {
            // prepared requests that can never be admitted any more
            for (int64_t id : prepared) {
                Req *r = reqs[id].get();
                if (r->H) hmat_free_synced(r->H);
                if (r->M) mesh_free_synced(r->M);
                r->H = nullptr;
                r->M = nullptr;
                r->state = BEM_REQ_CANCELLED;
                r->status = BEM_E_STATE;
                ++cancelled;
            }
            prepared.clear();
            cv_done.notify_all();
            break;
        }
        // poll in-flight batches often; otherwise sleep until notified
        cv_engine.wait_for(lk, any_inflight || !admitted.empty()
                                   ? std::chrono::microseconds(100)
                                   : std::chrono::microseconds(20000));
    }
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
        for (int s = 0; s < kEngineStreams; ++s) {
            if (cudaStreamCreateWithFlags(&S->streams[s], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&S->events[s], cudaEventDisableTiming) != cudaSuccess) {
                set_last_error("cannot create the engine streams");
                for (int q = 0; q <= s; ++q) {
                    if (S->streams[q]) cudaStreamDestroy(S->streams[q]);
                    if (S->events[q]) cudaEventDestroy(S->events[q]);
                }
                return BEM_E_CUDA;
            }
        }
    }
    for (int i = 0; i < max_slots; ++i) S->workers.emplace_back([s = S.get()] { s->worker(); });
    S->engine = std::thread([s = S.get()] { s->engine_loop(); });
    *out = S.release();
    return BEM_OK;
}

int bem_server_submit(bem_server S, const bem_request *q, int64_t *req_id)
{
    if (!S || !q || !req_id) return BEM_E_ARG;
    const bool product = q->reuse > 0;
    if (!q->x || (!product && (!q->vertices || !q->triangles || q->n_vertices < 3 ||
                               q->n_triangles < 1 || q->op < 0 || q->op > 2 ||
                               (q->prec != BEM_FP64 && q->prec != BEM_MIXED && q->prec != BEM_MIXED_SP) ||
                               !(q->aca_eps > 0) || q->leaf_size < 1 || !(q->eta > 0))) ||
        (product && q->n_triangles < 1)) {
        set_last_error("bad request");
        return BEM_E_ARG;
    }
    auto r = std::make_unique<Req>();
    r->reuse = product ? q->reuse : 0;
    if (!product) {
        r->V.assign(q->vertices, q->vertices + 3 * q->n_vertices);
        r->T.assign(q->triangles, q->triangles + 3 * q->n_triangles);
    }
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
    if (product && !S->find_resident(q->reuse) && S->reqs.find(q->reuse) == S->reqs.end()) {
        set_last_error("the request to reuse has no resident matrix");
        return BEM_E_STATE;
    }
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
    info->launch_requests = r.launch_reqs;
    info->reused = r.reused;
    info->t_ready_ms = r.t_ready;
    info->t_launch_ms = r.t_launch;
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
    // the matrix, if resident, is kept apart from the record (reuse names
    // the request's id)
    S->reqs.erase(it);
    return status;
}

int bem_server_cancel(bem_server S, int64_t id)
{
    if (!S) return BEM_E_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return BEM_E_ARG;
    Req *r = it->second.get();
    auto q = std::find(S->queue.begin(), S->queue.end(), id);
    if (q != S->queue.end()) {
        S->queue.erase(q);
    } else {
        auto p = std::find(S->prepared.begin(), S->prepared.end(), id);
        if (p != S->prepared.end()) {
            S->prepared.erase(p);
            if (r->H) hmat_free_synced(r->H);
            if (r->M) mesh_free_synced(r->M);
            r->H = nullptr;
            r->M = nullptr;
        } else if (r->state == BEM_REQ_PREPARING) {
            // the worker frees its host objects when it sees the state
        } else {
            return BEM_E_STATE;   // admitted: it runs to completion
        }
    }
    r->state = BEM_REQ_CANCELLED;
    r->status = BEM_E_STATE;
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
    out->queued = (int64_t)S->queue.size() + (int64_t)S->prepared.size() + S->preparing;
    out->running = S->running;
    out->reserved_bytes = S->in_use;
    out->peak_reserved_bytes = S->peak;
    out->budget_bytes = S->budget;
    out->resident = (int64_t)S->residents.size();
    out->resident_bytes = 0;
    for (const Resident &R : S->residents) out->resident_bytes += R.bytes;
    out->evictions = S->evictions;
    out->reuse_hits = S->reuse_hits;
    out->aca_launches = S->fused_launches;
    out->aca_launch_requests = S->fused_requests;
    out->max_launch_requests = S->max_launch_requests;
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
        S->cv_engine.notify_all();
        S->cv_done.notify_all();
    }
    for (auto &t : S->workers) t.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->cv_engine.notify_all();
    }
    if (S->engine.joinable()) S->engine.join();
    if (!(S->flags & BEM_SERVER_DRY_RUN)) cudaSetDevice(S->device);
    for (Resident &R : S->residents) {
        if (R.H) hmat_free_synced(R.H);
        if (R.M) mesh_free_synced(R.M);
    }
    S->residents.clear();
    for (int s = 0; s < kEngineStreams; ++s) {
        if (S->streams[s]) cudaStreamDestroy(S->streams[s]);
        if (S->events[s]) cudaEventDestroy(S->events[s]);
        if (S->staging[s]) cudaFreeHost(S->staging[s]);
    }
    delete S;
    return BEM_OK;
}

}  // extern "C"
