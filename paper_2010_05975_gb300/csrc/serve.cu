// Serving runtime: continuous batching of linear-solve requests on one GPU.
// (The paper has no serving layer; this is the request loop around its
// factorization: the mixed-precision LU + binary64 refinement of ir.cu.)
//
//   serve_enqueue  copies the request (A, B) into host memory, checks that it
//                  can ever fit the HBM budget, queues it, returns a ticket.
//   workers        one host thread + one CUDA stream per slot.  A free slot
//                  admits the first queued request whose device memory fits
//                  the budget (evicting unused cached factors, oldest first,
//                  when that makes room), so requests that arrive while
//                  others run start as soon as a slot and memory free up,
//                  and their kernels overlap on the device.
//   factor cache   requests with a nonzero matrix_id leave their binary64 A
//                  and low-precision factors on the device; a later request
//                  with the same id skips the copy of A and the factorization.
//   serve_poll     non-blocking status; copies X out once the request is done.
//
// Every request runs the same deterministic kernels on its own stream, so its
// result does not depend on what else is in flight.
#include "common.cuh"
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace lu {
namespace srv {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket = 0;
    int n = 0, nrhs = 0, flags = 0, precision = 0;
    uint64_t matrix_id = 0;
    double tol = 1e-12;
    std::vector<double> A, B, X;
    bool borrow = false, dev_in = false;     // borrow: read the caller's buffers in place
    const double* bA = nullptr;
    const double* bB = nullptr;
    int blda = 0, bldb = 0;
    int status = SERVE_PENDING;
    int error = 0;
    int cache_hit = 0;
    ir_result res{};
    size_t transient = 0, persistent = 0;   // bytes charged while running
    Clock::time_point t_enq, t_start, t_done;
};

struct Entry {
    uint64_t id = 0;
    int n = 0;
    double* A64 = nullptr;
    IrFactors fac{};
    size_t bytes = 0;
    int pins = 0;
    uint64_t last_use = 0;
};

class Server {
  public:
    explicit Server(const serve_cfg& c) : cfg_(c) {}
    int start();
    void shutdown();
    int enqueue(const serve_req& r, uint64_t* ticket);
    int poll(uint64_t ticket, serve_status* st, double* X);
    void stats(serve_stats* out);

  private:
    size_t persistent_bytes(int n) const {
        return static_cast<size_t>(n) * n * (8 + 4) + static_cast<size_t>(n) * 4 + 4096;
    }
    size_t transient_bytes(int n, int nrhs) const {
        // B, X, the refinement workspace, and the factorization's and solve's
        // own scratch (quantized panels, diagonal-block inverses: ~2 KB per row)
        return 2 * static_cast<size_t>(n) * nrhs * 8 + ir_workspace_bytes(n, nrhs, 30) + static_cast<size_t>(n) * 2048;
    }
    bool try_admit(Req* r, cudaStream_t s);     // caller holds mu_
    void evict_for(size_t need, cudaStream_t s);    // caller holds mu_
    void free_entry(Entry& e, cudaStream_t s);
    void worker(int slot);
    void run(Req* r, cudaStream_t s);

    serve_cfg cfg_;
    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<Req*> queue_;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs_;
    std::unordered_map<uint64_t, Entry> cache_;
    std::vector<std::thread> workers_;
    size_t used_ = 0, peak_ = 0;
    uint64_t next_ticket_ = 1, clock_ = 0;
    long long done_ = 0, failed_ = 0, hits_ = 0, evictions_ = 0;
    int running_ = 0, peak_running_ = 0;
    bool stop_ = false;
    int device_ = 0;
};

int Server::start() {
    if (!cfg_.dry_run) {
        if (cudaGetDevice(&device_) != cudaSuccess) {
            cudaGetLastError();
            return LU_ELAUNCH;
        }
    }
    const int slots = cfg_.max_slots > 0 ? cfg_.max_slots : 4;
    for (int i = 0; i < slots; ++i) workers_.emplace_back(&Server::worker, this, i);
    return 0;
}

void Server::shutdown() {
    {
        std::lock_guard<std::mutex> lk(mu_);
        stop_ = true;
        for (Req* r : queue_) {
            r->status = SERVE_FAILED;
            r->error = LU_EBUSY;
        }
        queue_.clear();
    }
    cv_.notify_all();
    for (auto& t : workers_) t.join();
    workers_.clear();
    for (auto& kv : cache_) free_entry(kv.second, nullptr);
    if (!cfg_.dry_run) cudaDeviceSynchronize();
    cache_.clear();
}

int Server::enqueue(const serve_req& q, uint64_t* ticket) {
    if (q.n < 1) return -2;
    if (q.nrhs < 1 || q.nrhs > 64) return -2;
    if (q.A == nullptr || q.lda < q.n) return -2;
    if (q.B == nullptr || q.ldb < q.nrhs) return -2;
    if (ticket == nullptr) return -3;
    auto r = std::make_unique<Req>();
    r->n = q.n;
    r->nrhs = q.nrhs;
    r->flags = q.flags;
    r->precision = q.precision ? q.precision : (cfg_.precision ? cfg_.precision : LU_PREC_BF16);
    r->matrix_id = q.matrix_id;
    r->tol = q.tol > 0.0 ? q.tol : (cfg_.tol > 0.0 ? cfg_.tol : 1e-12);
    r->persistent = persistent_bytes(q.n);
    r->transient = transient_bytes(q.n, q.nrhs);
    if (r->persistent + r->transient > cfg_.hbm_budget_bytes) return LU_EBUSY;   // can never fit
    r->borrow = (q.flags & SERVE_FLAG_BORROW) != 0;
    r->dev_in = q.device_inputs != 0;
    if (r->borrow) {
        r->bA = q.A;
        r->bB = q.B;
        r->blda = q.lda;
        r->bldb = q.ldb;
    } else {
        r->A.resize(static_cast<size_t>(q.n) * q.n);
        r->B.resize(static_cast<size_t>(q.n) * q.nrhs);
        if (q.device_inputs && !cfg_.dry_run) {
            if (cudaMemcpy2D(r->A.data(), sizeof(double) * q.n, q.A, sizeof(double) * q.lda, sizeof(double) * q.n,
                             q.n, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy2D(r->B.data(), sizeof(double) * q.nrhs, q.B, sizeof(double) * q.ldb,
                             sizeof(double) * q.nrhs, q.n, cudaMemcpyDeviceToHost) != cudaSuccess) {
                cudaGetLastError();
                return LU_ELAUNCH;
            }
        } else if (!q.device_inputs) {
            for (int i = 0; i < q.n; ++i) {
                std::memcpy(&r->A[static_cast<size_t>(i) * q.n], q.A + static_cast<size_t>(i) * q.lda,
                            sizeof(double) * q.n);
                std::memcpy(&r->B[static_cast<size_t>(i) * q.nrhs], q.B + static_cast<size_t>(i) * q.ldb,
                            sizeof(double) * q.nrhs);
            }
        }
    }
    r->t_enq = Clock::now();
    std::lock_guard<std::mutex> lk(mu_);
    if (stop_) return LU_EBUSY;
    if (cfg_.max_queue > 0 && static_cast<int>(queue_.size()) >= cfg_.max_queue) return LU_EBUSY;
    r->ticket = next_ticket_++;
    *ticket = r->ticket;
    queue_.push_back(r.get());
    reqs_.emplace(r->ticket, std::move(r));
    cv_.notify_one();
    return 0;
}

void Server::free_entry(Entry& e, cudaStream_t s) {
    if (cfg_.dry_run) return;
    if (e.A64) cudaFreeAsync(e.A64, s);
    ir_release(&e.fac, s);
    e.A64 = nullptr;
}

// Unused cached factors go, least recently used first, until `need` fits.
void Server::evict_for(size_t need, cudaStream_t s) {
    while (used_ + need > cfg_.hbm_budget_bytes) {
        auto victim = cache_.end();
        for (auto it = cache_.begin(); it != cache_.end(); ++it)
            if (it->second.pins == 0 && (victim == cache_.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == cache_.end()) return;
        free_entry(victim->second, s);
        used_ -= victim->second.bytes;
        ++evictions_;
        cache_.erase(victim);
    }
}

bool Server::try_admit(Req* r, cudaStream_t s) {
    auto it = (r->matrix_id != 0) ? cache_.find(r->matrix_id) : cache_.end();
    const bool hit = (it != cache_.end() && it->second.n == r->n);
    if (hit && it->second.pins > 0) return false;            // one request per cached matrix at a time
    const size_t need = r->transient + (hit ? 0 : r->persistent);
    if (used_ + need > cfg_.hbm_budget_bytes) {
        if (hit) it->second.pins += 1;                       // keep its own entry out of the eviction
        evict_for(need, s);
        if (hit) it->second.pins -= 1;
        if (used_ + need > cfg_.hbm_budget_bytes) return false;
    }
    used_ += need;
    if (used_ > peak_) peak_ = used_;
    r->cache_hit = hit ? 1 : 0;
    if (hit) {
        it->second.pins += 1;
        it->second.last_use = ++clock_;
        r->persistent = 0;
    }
    return true;
}

void Server::worker(int slot) {
    (void)slot;
    cudaStream_t s = nullptr;
    if (!cfg_.dry_run) {
        cudaSetDevice(device_);
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            s = nullptr;
        }
    }
    for (;;) {
        Req* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu_);
            for (;;) {
                if (stop_) break;
                for (auto it = queue_.begin(); it != queue_.end(); ++it)
                    if (try_admit(*it, s)) {
                        r = *it;
                        queue_.erase(it);
                        break;
                    }
                if (r) break;
                cv_.wait(lk);
            }
            if (!r) break;
            r->status = SERVE_RUNNING;
            r->t_start = Clock::now();
            ++running_;
            if (running_ > peak_running_) peak_running_ = running_;
        }
        run(r, s);
        {
            std::lock_guard<std::mutex> lk(mu_);
            --running_;
            r->t_done = Clock::now();
            used_ -= r->transient;
            if (r->status == SERVE_DONE) ++done_;
            else ++failed_;
            if (r->cache_hit) ++hits_;
        }
        cv_.notify_all();
    }
    if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
}

// One request on one stream.  Device memory: A64 and the factors (kept in
// the cache when matrix_id != 0), B64, X64 and the refinement workspace.
void Server::run(Req* r, cudaStream_t s) {
    const int n = r->n, nr = r->nrhs;
    if (cfg_.dry_run) {
        // scheduler test mode: no device work; the request holds its budget
        // for a time proportional to its flops, then reports its flags
        const double secs = 1.5e-10 * static_cast<double>(n) * n * n + 1e-4;
        std::this_thread::sleep_for(std::chrono::duration<double>(secs));
        std::lock_guard<std::mutex> lk(mu_);
        const bool fail = (r->flags & SERVE_FLAG_FAIL) != 0;
        r->status = fail ? SERVE_FAILED : SERVE_DONE;
        r->error = fail ? LU_ELAUNCH : 0;
        r->res.eta = -1.0;
        r->res.path = -1;
        if (r->cache_hit) {
            Entry& e = cache_[r->matrix_id];
            e.pins -= 1;
            e.last_use = ++clock_;
            return;
        }
        if (!fail && r->matrix_id != 0 && cache_.find(r->matrix_id) == cache_.end()) {
            Entry e;
            e.id = r->matrix_id;
            e.n = n;
            e.bytes = r->persistent;
            e.last_use = ++clock_;
            cache_.emplace(e.id, e);
        } else {
            used_ -= r->persistent;
        }
        return;
    }
    int rc = 0;
    double* A64 = nullptr;
    double* B64 = nullptr;
    double* X64 = nullptr;
    IrFactors fac{};
    Entry* hit = nullptr;
    if (r->cache_hit) {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = cache_.find(r->matrix_id);
        hit = &it->second;
        A64 = hit->A64;
        fac = hit->fac;
    }
    const size_t nn = static_cast<size_t>(n) * n;
    const cudaMemcpyKind kin = r->dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const double* Ause = A64;
    int ldu = n;
    if (!hit) {
        if (r->borrow && r->dev_in) {
            Ause = r->bA;                                     // the caller's device matrix, read in place
            ldu = r->blda;
        } else {
            if (cudaMallocAsync(reinterpret_cast<void**>(&A64), nn * sizeof(double), s) != cudaSuccess) rc = LU_ENOMEM;
            if (!rc) {
                const cudaError_t e =
                    r->borrow ? cudaMemcpy2DAsync(A64, sizeof(double) * n, r->bA, sizeof(double) * r->blda,
                                                  sizeof(double) * n, n, kin, s)
                              : cudaMemcpyAsync(A64, r->A.data(), nn * sizeof(double), cudaMemcpyHostToDevice, s);
                if (e != cudaSuccess) rc = LU_ELAUNCH;
            }
            Ause = A64;
        }
    }
    if (!rc && (cudaMallocAsync(reinterpret_cast<void**>(&B64), sizeof(double) * n * nr, s) != cudaSuccess ||
                cudaMallocAsync(reinterpret_cast<void**>(&X64), sizeof(double) * n * nr, s) != cudaSuccess))
        rc = LU_ENOMEM;
    if (!rc) {
        const cudaError_t e =
            r->borrow ? cudaMemcpy2DAsync(B64, sizeof(double) * nr, r->bB, sizeof(double) * r->bldb,
                                          sizeof(double) * nr, n, kin, s)
                      : cudaMemcpyAsync(B64, r->B.data(), sizeof(double) * n * nr, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) rc = LU_ELAUNCH;
    }
    if (!rc && !hit) rc = ir_factor(n, Ause, ldu, r->precision, 128, 128, &fac, s);
    ir_opts o{};
    o.precision = r->precision;
    o.tol = r->tol;
    if (!rc) rc = ir_refine(&fac, Ause, ldu, nr, B64, nr, X64, nr, &o, &r->res, s);
    if (!rc) {
        r->X.resize(static_cast<size_t>(n) * nr);
        if (cudaMemcpyAsync(r->X.data(), X64, sizeof(double) * n * nr, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            rc = LU_ELAUNCH;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = LU_ELAUNCH;
    cudaGetLastError();
    if (B64) cudaFreeAsync(B64, s);
    if (X64) cudaFreeAsync(X64, s);
    std::lock_guard<std::mutex> lk(mu_);
    const bool ok = (rc == 0 && r->res.path >= 0 && r->res.info == 0);
    r->status = ok ? SERVE_DONE : SERVE_FAILED;
    r->error = rc ? rc : (ok ? 0 : (r->res.info != 0 ? LU_EUNSUPPORTED : LU_ETIMEOUT));
    if (hit) {
        hit->fac = fac;                                       // the ladder may have refactored
        hit->pins -= 1;
        hit->last_use = ++clock_;
        return;
    }
    bool keep = ok && r->matrix_id != 0 && cache_.find(r->matrix_id) == cache_.end();
    if (keep && A64 == nullptr) {
        // a borrowed device matrix: the cache keeps its own copy
        if (cudaMallocAsync(reinterpret_cast<void**>(&A64), nn * sizeof(double), s) != cudaSuccess ||
            cudaMemcpy2DAsync(A64, sizeof(double) * n, Ause, sizeof(double) * ldu, sizeof(double) * n, n,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            keep = false;
        }
    }
    if (keep) {
        Entry e;
        e.id = r->matrix_id;
        e.n = n;
        e.A64 = A64;
        e.fac = fac;
        e.bytes = r->persistent;
        e.last_use = ++clock_;
        cache_.emplace(e.id, e);
    } else {
        if (A64) cudaFreeAsync(A64, s);
        ir_release(&fac, s);
        cudaStreamSynchronize(s);
        used_ -= r->persistent;
    }
}

int Server::poll(uint64_t ticket, serve_status* st, double* X) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = reqs_.find(ticket);
    if (it == reqs_.end()) return LU_ENOTFOUND;
    Req* r = it->second.get();
    *st = serve_status{};
    st->status = r->status;
    st->error = r->error;
    st->cache_hit = r->cache_hit;
    st->eta = r->res.eta;
    st->iters = r->res.iters;
    st->gmres_iters = r->res.gmres_iters;
    st->path = r->res.path;
    st->precision = r->res.precision;
    if (r->status == SERVE_DONE || r->status == SERVE_FAILED) {
        st->queue_s = std::chrono::duration<double>(r->t_start - r->t_enq).count();
        st->latency_s = std::chrono::duration<double>(r->t_done - r->t_enq).count();
        if (r->status == SERVE_DONE && X && !r->X.empty()) std::memcpy(X, r->X.data(), sizeof(double) * r->X.size());
        reqs_.erase(it);
    }
    return 0;
}

void Server::stats(serve_stats* out) {
    std::lock_guard<std::mutex> lk(mu_);
    *out = serve_stats{};
    out->budget_bytes = cfg_.hbm_budget_bytes;
    out->used_bytes = used_;
    out->peak_bytes = peak_;
    out->queued = static_cast<int>(queue_.size());
    out->running = running_;
    out->peak_running = peak_running_;
    out->completed = done_;
    out->failed = failed_;
    out->cache_hits = hits_;
    out->cache_entries = static_cast<int>(cache_.size());
    out->evictions = evictions_;
}

}  // namespace srv
}  // namespace lu

struct serve_t {
    lu::srv::Server* s;
};

extern "C" int serve_create(const serve_cfg* cfg, serve_t** h) {
    if (cfg == nullptr) return -1;
    if (h == nullptr) return -2;
    if (cfg->hbm_budget_bytes == 0 || cfg->max_slots < 0 || cfg->max_slots > 64) return -1;
    auto* srv = new lu::srv::Server(*cfg);
    if (int rc = srv->start()) {
        delete srv;
        return rc;
    }
    *h = new serve_t{srv};
    return 0;
}

extern "C" int serve_enqueue(serve_t* h, const serve_req* r, uint64_t* ticket) {
    if (h == nullptr) return -1;
    if (r == nullptr) return -2;
    return h->s->enqueue(*r, ticket);
}

extern "C" int serve_poll(serve_t* h, uint64_t ticket, serve_status* st, double* X) {
    if (h == nullptr) return -1;
    if (st == nullptr) return -3;
    return h->s->poll(ticket, st, X);
}

extern "C" int serve_get_stats(serve_t* h, serve_stats* out) {
    if (h == nullptr) return -1;
    if (out == nullptr) return -2;
    h->s->stats(out);
    return 0;
}

extern "C" int serve_destroy(serve_t* h) {
    if (h == nullptr) return -1;
    h->s->shutdown();
    delete h->s;
    delete h;
    return 0;
}
