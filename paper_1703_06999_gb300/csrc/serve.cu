// Serving loop: evaluations of different grids arrive over time; each is
// admitted when its device-memory footprint fits the server's budget,
// planned on a host thread, and joins the next batched launch (one launch
// per stage over all systems of the batch).  Up to max_inflight batches run
// at once on their own streams, so requests that arrive while others are on
// the GPU are admitted and overlap with them (continuous batching).  The
// kernel table stays resident on the device for the server's lifetime, and
// so do plans: a finished request's handle (buffers, FFT twiddles, tile
// shapes, tensor maps) stays on the device, counted against the pool, and
// the next request of the same grid re-plans only what depends on its cell
// and functional (metric and k-point order, sorted on the device).  Idle
// plans are evicted, least recently used first, when an admission needs
// their memory.
#include <algorithm>
#include <atomic>
#include <list>
#include <tuple>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace vdwgb;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    long long id = 0;
    int functional = 1;
    int nx = 0, ny = 0, nz = 0;
    double cell[9];
    const double *rho = nullptr, *sigma = nullptr;
    double *dedrho = nullptr, *dedsigma = nullptr;
    double t_submit = 0, t_done = 0;
    double energy = 0;
    int status = 1;              // 1 pending, 0 done, < 0 error code (published under the lock)
    int err = 0;                 // launch error noted by the dispatcher, published by the completer
    size_t footprint = 0;
    size_t npts = 0;
    vdwgb_data *h = nullptr;
    cudaEvent_t ready = nullptr;  // planning + input upload finished
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    SysDev *hdesc = nullptr;     // pinned host staging of the launch descriptors
    int *hpre = nullptr;
    SysDev *ddesc = nullptr;
    int *dpre = nullptr;
    double *denergy = nullptr;
    double *henergy = nullptr;   // pinned
    std::vector<Req *> reqs;
    bool busy = false;
};

}  // namespace

struct vdwgb_server_s {
    int device = 0, prec = 1, max_batch = 8, max_inflight = 2, nplan = 8;   // nplan: planner threads
    // requests taken by a planner and not yet dispatched, and their bound:
    // the rest wait on the host, holding no device memory, so that idle
    // resident plans are not evicted for requests that cannot run yet
    int staged = 0, max_staged = 0;
    size_t pool = 0, used = 0, peak = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> pending, ready;
    std::unordered_map<long long, Req *> reqs;
    std::vector<Slot> slots;
    std::vector<cudaStream_t> plan_streams;
    std::vector<std::thread> workers;
    bool stop = false;
    long long next_id = 1;
    // resident plans not in use, most recently used first: (grid, handle, footprint)
    struct Idle {
        std::tuple<int, int, int> grid;
        vdwgb_data *h;
        size_t footprint;
    };
    std::list<Idle> idle;
    long long plans_reused = 0, plans_built = 0;
    // statistics
    long long submitted = 0, completed = 0, failed = 0, batches = 0, batched_reqs = 0;
    double t_first = 0, t_last = 0;
    double pts_done = 0;
    std::vector<double> lat;
};

static size_t request_footprint(int nx, int ny, int nz, int prec) {
    const size_t N = (size_t)nx * ny * nz;
    return vdwgb_footprint_bytes(nx, ny, nz, prec) + (4 * N + 1) * sizeof(double) + (1u << 20);
}

// an idle resident plan of this grid, or nullptr (under the lock); one of
// the same cell first (its re-plan skips the k-point sort)
static vdwgb_data *take_idle(vdwgb_server_s *s, const Req *r) {
    const auto key = std::make_tuple(r->nx, r->ny, r->nz);
    auto pick = s->idle.end();
    for (auto it = s->idle.begin(); it != s->idle.end(); ++it) {
        if (it->grid != key) continue;
        if (std::memcmp(it->h->cell, r->cell, sizeof r->cell) == 0) {
            pick = it;
            break;
        }
        if (pick == s->idle.end()) pick = it;
    }
    if (pick == s->idle.end()) return nullptr;
    vdwgb_data *h = pick->h;
    s->idle.erase(pick);
    return h;
}

static size_t idle_bytes(const vdwgb_server_s *s) {
    size_t b = 0;
    for (const auto &x : s->idle) b += x.footprint;
    return b;
}

// planner: admit in arrival order while the footprint fits (a resident plan
// of the same grid, the free pool, or the free pool after evicting idle
// plans), plan or re-plan, upload inputs
static void planner_loop(vdwgb_server_s *s, int k) {
    cudaSetDevice(s->device);
    cudaStream_t st = s->plan_streams[k];
    for (;;) {
        Req *r = nullptr;
        vdwgb_data *reuse = nullptr;
        std::vector<vdwgb_data *> evict;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                if (s->stop) return true;
                if (s->pending.empty() || s->staged >= s->max_staged) return false;
                const Req *f = s->pending.front();
                const auto key = std::make_tuple(f->nx, f->ny, f->nz);
                for (const auto &x : s->idle)
                    if (x.grid == key) return true;
                return f->footprint <= s->pool - s->used + idle_bytes(s);
            });
            if (s->stop) return;
            r = s->pending.front();
            s->pending.pop_front();
            ++s->staged;
            reuse = take_idle(s, r);
            if (reuse) {
                ++s->plans_reused;             // its footprint stays counted in used
            } else {
                while (r->footprint > s->pool - s->used && !s->idle.empty()) {
                    evict.push_back(s->idle.back().h);   // least recently used
                    s->used -= s->idle.back().footprint;
                    s->idle.pop_back();
                }
                s->used += r->footprint;
                ++s->plans_built;
            }
            s->peak = std::max(s->peak, s->used);
        }
        for (vdwgb_data *h : evict) vdwgb_finalize(&h);   // stream-ordered frees
        int rc = 0;
        if (reuse) {
            r->h = reuse;
            r->h->alloc_stream = st;           // this planner's stream orders its work from now on
            rc = handle_replan(r->h, r->cell, r->functional);
        } else {
            rc = vdwgb_new(r->functional, &r->h);
            if (!rc)
                rc = vdwgb_set_unit_cell(r->h, r->nx, r->ny, r->nz, r->cell[0], r->cell[1], r->cell[2], r->cell[3],
                                         r->cell[4], r->cell[5], r->cell[6], r->cell[7], r->cell[8]);
            if (!rc) rc = handle_init(r->h, s->device, s->prec, st);
        }
        if (!rc) {
            const size_t N = r->npts;
            cudaError_t e = cudaMemcpyAsync(r->h->d_io, r->rho, N * sizeof(double), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(r->h->d_io + N, r->sigma, N * sizeof(double), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(r->ready, st);
            if (e != cudaSuccess) rc = cuda_fail(e, "request upload");
        }
        std::lock_guard<std::mutex> lk(s->mu);
        if (rc) {
            if (r->h) vdwgb_finalize(&r->h);
            s->used -= r->footprint;
            --s->staged;
            r->status = rc;
            r->t_done = now_s();
            ++s->failed;
        } else {
            s->ready.push_back(r);
        }
        s->cv.notify_all();
    }
}

// dispatcher: whenever a slot is free, launch everything that is ready (up to
// max_batch) as one batch on that slot's stream
static void dispatcher_loop(vdwgb_server_s *s) {
    cudaSetDevice(s->device);
    for (;;) {
        Slot *slot = nullptr;
        std::vector<Req *> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                if (s->stop) return true;
                if (s->ready.empty()) return false;
                for (auto &sl : s->slots)
                    if (!sl.busy) return true;
                return false;
            });
            if (s->stop) return;
            for (auto &sl : s->slots)
                if (!sl.busy) {
                    slot = &sl;
                    break;
                }
            while (!s->ready.empty() && (int)batch.size() < s->max_batch) {
                batch.push_back(s->ready.front());
                s->ready.pop_front();
                --s->staged;
            }
            slot->busy = true;
        }
        const int n = (int)batch.size();
        std::vector<vdwgb_data *> hs(n);
        for (int i = 0; i < n; ++i) hs[i] = batch[i]->h;
        LaunchSet L;
        int rc = batch_launchset(hs.data(), n, slot->hdesc, slot->hpre, slot->ddesc, slot->dpre, L);
        cudaError_t e = cudaSuccess;
        if (!rc) {
            for (int i = 0; i < n; ++i) {
                const size_t N = batch[i]->npts;
                double *d = hs[i]->d_io;
                SysDev &D = slot->hdesc[i];
                D.n = d;
                D.sigma = d + N;
                D.dedn = d + 2 * N;
                D.dedsigma = d + 3 * N;
                D.energy = slot->denergy + i;
                e = cudaStreamWaitEvent(slot->st, batch[i]->ready, 0);
                if (e != cudaSuccess) break;
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(slot->ddesc, slot->hdesc, n * sizeof(SysDev), cudaMemcpyHostToDevice, slot->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(slot->dpre, slot->hpre, NKIND * (n + 1) * sizeof(int), cudaMemcpyHostToDevice,
                                    slot->st);
            if (e == cudaSuccess) e = launch_all(L, s->prec, slot->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(slot->henergy, slot->denergy, n * sizeof(double), cudaMemcpyDeviceToHost,
                                    slot->st);
            if (e == cudaSuccess) e = cudaEventRecord(slot->done, slot->st);
            if (e != cudaSuccess) rc = cuda_fail(e, "batch launch");
        }
        std::lock_guard<std::mutex> lk(s->mu);
        slot->reqs = batch;
        if (rc) {
            // fail the whole batch; its slot is released by the completer
            for (Req *r : batch) r->err = rc;
        }
        ++s->batches;
        s->batched_reqs += n;
        s->cv.notify_all();
    }
}

// completer: poll the busy slots; for each finished batch copy the results
// back, release the requests' memory and free the slot
static void complete_slot(vdwgb_server_s *s, Slot *slot, int dev_rc, cudaStream_t cst) {
    std::vector<Req *> reqs;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        reqs = slot->reqs;
    }
    // results are copied outside the lock; a request is published as done
    // only under the lock (a waiting caller may free it right after)
    std::vector<int> st(reqs.size());
    std::vector<double> en(reqs.size(), 0.0);
    std::vector<int> pend(reqs.size());
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t i = 0; i < reqs.size(); ++i) pend[i] = reqs[i]->err ? reqs[i]->err : reqs[i]->status;
    }
    // every copy of the batch first, then one wait: the copies run back to back
    cudaError_t ce = cudaSuccess;
    if (dev_rc == 0) {
        for (size_t i = 0; i < reqs.size() && ce == cudaSuccess; ++i) {
            if (pend[i] != 1) continue;
            Req *r = reqs[i];
            const size_t N = r->npts;
            ce = cudaMemcpyAsync(r->dedrho, r->h->d_io + 2 * N, N * sizeof(double), cudaMemcpyDeviceToHost, cst);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(r->dedsigma, r->h->d_io + 3 * N, N * sizeof(double), cudaMemcpyDeviceToHost, cst);
        }
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(cst);
    }
    for (size_t i = 0; i < reqs.size(); ++i) {
        Req *r = reqs[i];
        const int pending_status = pend[i];
        if (pending_status == 1 && dev_rc == 0) {
            en[i] = slot->henergy[i];
            st[i] = ce == cudaSuccess ? 0 : VDWGB_ECUDA;
        } else if (pending_status == 1) {
            st[i] = dev_rc ? dev_rc : VDWGB_ECUDA;
        } else {
            st[i] = pending_status;
        }
        if (r->ready) cudaEventDestroy(r->ready);
        r->ready = nullptr;
        // failed requests release their plan (stream-ordered frees); finished
        // ones keep it resident for the next request of the same grid
        if (r->h && st[i] != 0) vdwgb_finalize(&r->h);
    }
    const double t = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < reqs.size(); ++i) {
        Req *r = reqs[i];
        r->energy = en[i];
        r->t_done = t;
        if (r->h) {
            s->idle.push_front({std::make_tuple(r->nx, r->ny, r->nz), r->h, r->footprint});
            r->h = nullptr;
        } else {
            s->used -= r->footprint;
        }
        if (st[i] == 0) {
            ++s->completed;
            s->pts_done += (double)r->npts;
            s->lat.push_back(r->t_done - r->t_submit);
        } else {
            ++s->failed;
        }
        s->t_last = t;
        r->status = st[i];
    }
    slot->reqs.clear();
    slot->busy = false;
    s->cv.notify_all();
}

static void completer_loop(vdwgb_server_s *s) {
    cudaSetDevice(s->device);
    cudaStream_t cst;
    cudaStreamCreateWithFlags(&cst, cudaStreamNonBlocking);
    std::vector<double> since(s->slots.size(), 0.0);
    for (;;) {
        std::vector<Slot *> busy;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                if (s->stop) return true;
                for (auto &sl : s->slots)
                    if (sl.busy && !sl.reqs.empty()) return true;
                return false;
            });
            if (s->stop) break;
            for (auto &sl : s->slots)
                if (sl.busy && !sl.reqs.empty()) busy.push_back(&sl);
        }
        bool any = false;
        for (Slot *sl : busy) {
            const size_t k = (size_t)(sl - s->slots.data());
            if (since[k] == 0.0) since[k] = now_s();
            const cudaError_t q = cudaEventQuery(sl->done);
            int rc;
            if (q == cudaSuccess) {
                rc = vdwgb_device_status(s->device);
            } else if (q == cudaErrorNotReady) {
                if (now_s() - since[k] <= 120.0) continue;   // bounded wait
                rc = VDWGB_ETIMEDOUT;
            } else {
                rc = VDWGB_ECUDA;
            }
            complete_slot(s, sl, rc, cst);
            since[k] = 0.0;
            any = true;
        }
        if (!any) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    cudaStreamDestroy(cst);
}

extern "C" {

int vdwgb_server_new(int device, int precision, size_t pool_bytes, int max_batch, int max_inflight,
                     vdwgb_server *out) {
    if (!out) return fail(VDWGB_EINVAL, "null output");
    *out = nullptr;
    if (precision != VDWGB_FP64 && precision != VDWGB_FP32_MIXED) return fail(VDWGB_EINVAL, "unknown precision");
    if (max_batch < 1 || max_batch > 256 || max_inflight < 1 || max_inflight > 8 || pool_bytes == 0)
        return fail(VDWGB_EINVAL, "max_batch 1..256, max_inflight 1..8, pool_bytes > 0");
    int rc = device_setup(device);
    if (rc) return rc;
    rc = vdwgb_kernel_table(device, nullptr, nullptr, nullptr);   // table resident before serving
    if (rc) return rc;
    cudaSetDevice(device);
    cudaMemPool_t mp;
    if (cudaDeviceGetDefaultMemPool(&mp, device) == cudaSuccess) {
        unsigned long long thr = ~0ull;   // keep freed blocks cached in the pool
        cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    vdwgb_server_s *s = new vdwgb_server_s();
    s->device = device;
    s->prec = precision;
    s->pool = pool_bytes;
    s->max_batch = max_batch;
    s->max_staged = max_batch * (max_inflight + 1);
    s->max_inflight = max_inflight;
    s->slots.resize(max_inflight);
    cudaError_t e = cudaSuccess;
    for (auto &sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.hdesc, max_batch * sizeof(SysDev));
        if (e == cudaSuccess) e = cudaMallocHost(&sl.hpre, NKIND * (max_batch + 1) * sizeof(int));
        if (e == cudaSuccess) e = cudaMallocHost(&sl.henergy, max_batch * sizeof(double));
        if (e == cudaSuccess) e = device_malloc(reinterpret_cast<void **>(&sl.ddesc), max_batch * sizeof(SysDev));
        if (e == cudaSuccess) e = device_malloc(reinterpret_cast<void **>(&sl.dpre), NKIND * (max_batch + 1) * sizeof(int));
        if (e == cudaSuccess) e = device_malloc(reinterpret_cast<void **>(&sl.denergy), max_batch * sizeof(double));
    }
    s->plan_streams.resize(s->nplan);
    for (auto &st : s->plan_streams)
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        vdwgb_server_free(&s);
        return cuda_fail(e, "server setup");
    }
    for (int k = 0; k < s->nplan; ++k) s->workers.emplace_back(planner_loop, s, k);
    s->workers.emplace_back(dispatcher_loop, s);
    s->workers.emplace_back(completer_loop, s);
    *out = s;
    return 0;
}

int vdwgb_server_submit(vdwgb_server s, int functional, int nx, int ny, int nz, const double *cell9,
                        const double *rho, const double *sigma, double *dedrho, double *dedsigma, long long *id) {
    if (!s || !cell9 || !rho || !sigma || !dedrho || !dedsigma || !id) return fail(VDWGB_EINVAL, "null argument");
    if (functional != VDWGB_DF1 && functional != VDWGB_DF2) return fail(VDWGB_EINVAL, "unknown functional");
    if (nx < 1 || ny < 1 || nz < 1) return fail(VDWGB_EINVAL, "bad grid");
    Req *r = new Req();
    r->functional = functional;
    r->nx = nx;
    r->ny = ny;
    r->nz = nz;
    std::memcpy(r->cell, cell9, sizeof r->cell);
    r->rho = rho;
    r->sigma = sigma;
    r->dedrho = dedrho;
    r->dedsigma = dedsigma;
    r->npts = (size_t)nx * ny * nz;
    r->footprint = request_footprint(nx, ny, nz, s->prec);
    if (r->footprint > s->pool) {
        delete r;
        return fail(VDWGB_EAGAIN, "request footprint %zu B exceeds the server pool", request_footprint(nx, ny, nz, s->prec));
    }
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->t_submit = now_s();
    if (s->submitted == 0) s->t_first = r->t_submit;
    ++s->submitted;
    s->reqs[r->id] = r;
    s->pending.push_back(r);
    *id = r->id;
    s->cv.notify_all();
    return 0;
}

int vdwgb_server_poll(vdwgb_server s, long long id, double *energy, double *latency_s) {
    if (!s) return fail(VDWGB_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(VDWGB_ENOTFOUND, "unknown request %lld", id);
    Req *r = it->second;
    if (r->status == 1) return 0;
    const int st = r->status;
    if (energy) *energy = r->energy;
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    s->reqs.erase(it);
    delete r;
    if (st < 0) return fail(st, "request %lld failed", id);
    return 1;
}

int vdwgb_server_wait(vdwgb_server s, long long id, double timeout_s, double *energy, double *latency_s) {
    if (!s) return fail(VDWGB_EINVAL, "null server");
    const double t0 = now_s();
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto it = s->reqs.find(id);
            if (it == s->reqs.end()) return fail(VDWGB_ENOTFOUND, "unknown request %lld", id);
            if (it->second->status == 1) {
                const double left = timeout_s - (now_s() - t0);
                if (left <= 0) return fail(VDWGB_ETIMEDOUT, "request %lld not done after %.3f s", id, timeout_s);
                s->cv.wait_for(lk, std::chrono::duration<double>(std::min(left, 0.05)));
                continue;
            }
        }
        return vdwgb_server_poll(s, id, energy, latency_s);
    }
}

int vdwgb_server_stats(vdwgb_server s, vdwgb_server_stats_t *out) {
    if (!s || !out) return fail(VDWGB_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->batches = s->batches;
    out->mean_batch = s->batches ? (double)s->batched_reqs / (double)s->batches : 0.0;
    out->pool_bytes = s->pool;
    out->pool_used_peak = s->peak;
    out->plans_reused = s->plans_reused;
    out->plans_built = s->plans_built;
    const double span = s->t_last - s->t_first;
    out->pts_per_s = span > 0 ? s->pts_done / span : 0.0;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        auto q = [&](double f) {
            size_t k = (size_t)(f * (double)(v.size() - 1) + 0.5);
            std::nth_element(v.begin(), v.begin() + k, v.end());
            return v[k];
        };
        out->p50_s = q(0.50);
        out->p99_s = q(0.99);
    }
    return 0;
}

int vdwgb_server_free(vdwgb_server *sp) {
    if (!sp) return fail(VDWGB_EINVAL, "null server pointer");
    vdwgb_server_s *s = *sp;
    if (!s) return 0;
    // let in-flight batches finish (bounded), then stop the workers
    const double t0 = now_s();
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            bool busy = false;
            for (auto &sl : s->slots) busy |= sl.busy;
            if (!busy || now_s() - t0 > 60.0) {
                s->stop = true;
                s->cv.notify_all();
                break;
            }
        }
        std::this_thread::sleep_for(std::chrono::milliseconds(2));
    }
    for (auto &t : s->workers) t.join();
    cudaSetDevice(s->device);
    for (auto &kv : s->reqs) {
        Req *r = kv.second;
        if (r->h) vdwgb_finalize(&r->h);
        if (r->ready) cudaEventDestroy(r->ready);
        delete r;
    }
    for (auto &x : s->idle) vdwgb_finalize(&x.h);
    s->idle.clear();
    for (auto &sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.done) cudaEventDestroy(sl.done);
        cudaFreeHost(sl.hdesc);
        cudaFreeHost(sl.hpre);
        cudaFreeHost(sl.henergy);
        cudaFree(sl.ddesc);
        cudaFree(sl.dpre);
        cudaFree(sl.denergy);
    }
    for (auto st : s->plan_streams) {
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    }
    delete s;
    *sp = nullptr;
    return 0;
}

}  // extern "C"
