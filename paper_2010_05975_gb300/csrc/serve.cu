// Serving runtime: continuous batching of linear-solve requests on one GPU.
// (The paper has no serving layer; this is the request loop around its
// factorization: the mixed-precision LU + binary64 refinement of ir.cu.)
//
//   serve_enqueue  copies the request (A, B) into host memory, checks that it
//                  can ever fit the HBM budget, queues it, returns a ticket.
//   workers        one host thread + one CUDA stream per slot.  A free slot
//                  admits the first queued large request whose device memory
//                  fits the budget (evicting unused cached factors, oldest
//                  first, when that makes room), so requests that arrive
//                  while others run start as soon as a slot and memory free
//                  up, and their kernels overlap on the device.
//   batch worker   one more thread + stream for the small requests (n up to
//                  batch_n_max): whenever it is free it admits every queued
//                  small request that fits the budget (up to batch_max) and
//                  solves them together, one launch per step for all of them
//                  (serve_batch.cu: binary32 batched factorization, binary64
//                  refinement).  Requests that arrive meanwhile form the
//                  next batch.  A small request whose refinement stops
//                  contracting is handed to a slot worker (the precision
//                  ladder of ir_solve).
//   factor cache   requests with a nonzero matrix_id leave their binary64 A
//                  and low-precision factors on the device; a later request
//                  with the same id skips the copy of A and the factorization.
//   serve_poll     non-blocking status; copies X out once the request is done.
//
// Every request runs the same deterministic kernels, whatever else shares
// its stream or its launches, so its result does not depend on what else is
// in flight.
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
    bool no_batch = false;                   // handed over from the batched path
    int batched = 0;                         // solved in a shared launch
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
    bool batched = false;      // binary32 factors of the batched path (no solve plan)
};

class Server {
  public:
    explicit Server(const serve_cfg& c) : cfg_(c) {}
    int start();
    void shutdown();
    int enqueue(const serve_req& r, uint64_t* ticket);
    int poll(uint64_t ticket, serve_status* st, double* X);
    void stats(serve_stats* out);

    // what a request keeps on the device when its factors are cached: A,
    // the binary32 factors and pivots, and (slot path) the solve plan's
    // diagonal-block inverses and coupling blocks (2 + 2 blocks of 128 x 128
    // floats per 128 rows, the last block padded) and permutation
    static size_t persistent_bytes(int n, bool batched) {
        const size_t nn = static_cast<size_t>(n) * n;
        size_t b = nn * (8 + 4) + static_cast<size_t>(n) * 4 + 4096;
        if (!batched) b += static_cast<size_t>((n + 127) / 128) * 128 * 2048 + static_cast<size_t>(n) * 4 + 4096;
        return b;
    }
    // what it needs only while it runs
    static size_t transient_bytes(int n, int nrhs, bool batched) {
        const size_t vs = static_cast<size_t>(n) * nrhs;
        if (batched) return vs * (3 * 8 + 4) + 16 * static_cast<size_t>(nrhs) + 4096;
        // B, X, the refinement workspace, the deferred quantized panels
        // (kDeferDefault slots of Lq, UqT: 2 x 256 x 2 bytes per row, plus
        // exponents) and the tournament's lists
        return 2 * vs * 8 + ir_workspace_bytes(n, nrhs, 30) +
               static_cast<size_t>(n) * (kDeferDefault * 1040 + 2048);
    }
  private:
    bool small(const Req* r) const { return bn_max_ > 0 && r->n <= bn_max_ && !r->no_batch; }
    bool try_admit(Req* r, cudaStream_t s);     // caller holds mu_
    void evict_for(size_t need, cudaStream_t s);    // caller holds mu_
    void free_entry(Entry& e, cudaStream_t s);
    void worker(int slot);
    void batch_worker();
    void run(Req* r, cudaStream_t s);
    void run_batch(std::vector<Req*>& rs, cudaStream_t s);
    void finish(Req* r);                         // caller holds mu_

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
    long long batches_ = 0, batched_ = 0;
    int queued_[2] = {0, 0};                   // queued requests per path: [0] slots, [1] shared batches
    bool stop_ = false;
    int device_ = 0;
    int bn_max_ = 1024, b_max_ = 256;
};

int Server::start() {
    if (!cfg_.dry_run) {
        if (cudaGetDevice(&device_) != cudaSuccess) {
            cudaGetLastError();
            return LU_ELAUNCH;
        }
    }
    bn_max_ = cfg_.batch_n_max == 0 ? 1024 : (cfg_.batch_n_max < 0 ? 0 : cfg_.batch_n_max);
    b_max_ = cfg_.batch_max > 0 ? cfg_.batch_max : 256;
    const int slots = cfg_.max_slots > 0 ? cfg_.max_slots : 4;
    for (int i = 0; i < slots; ++i) workers_.emplace_back(&Server::worker, this, i);
    if (bn_max_ > 0) workers_.emplace_back(&Server::batch_worker, this);
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
        queued_[0] = queued_[1] = 0;
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
    const bool sm = small(r.get());
    r->persistent = persistent_bytes(q.n, sm);
    r->transient = transient_bytes(q.n, q.nrhs, sm);
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
    // the queue bound holds per path, so a backlog of large requests does not
    // turn small ones away (and the reverse)
    if (cfg_.max_queue > 0 && queued_[sm ? 1 : 0] >= cfg_.max_queue) return LU_EBUSY;
    r->ticket = next_ticket_++;
    *ticket = r->ticket;
    ++queued_[sm ? 1 : 0];
    queue_.push_back(r.get());
    reqs_.emplace(r->ticket, std::move(r));
    cv_.notify_all();      // slot workers and the batch worker take different requests
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
    // cached factors serve the path that made them (the batched path keeps
    // binary32 factors without a solve plan)
    const bool hit = (it != cache_.end() && it->second.n == r->n && it->second.batched == small(r));
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
                    if (!small(*it) && try_admit(*it, s)) {
                        r = *it;
                        queue_.erase(it);
                        --queued_[0];
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
            finish(r);
        }
        cv_.notify_all();
    }
    if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
}

// The small requests: whenever this worker is free it admits every queued
// small request that fits the budget (up to b_max_) and solves them with
// shared launches.
void Server::batch_worker() {
    cudaStream_t s = nullptr;
    if (!cfg_.dry_run) {
        cudaSetDevice(device_);
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            s = nullptr;
        }
    }
    for (;;) {
        std::vector<Req*> rs;
        {
            std::unique_lock<std::mutex> lk(mu_);
            for (;;) {
                if (stop_) break;
                for (auto it = queue_.begin(); it != queue_.end() && static_cast<int>(rs.size()) < b_max_;) {
                    if (small(*it) && try_admit(*it, s)) {
                        rs.push_back(*it);
                        it = queue_.erase(it);
                        --queued_[1];
                    } else {
                        ++it;
                    }
                }
                if (!rs.empty()) break;
                cv_.wait(lk);
            }
            if (rs.empty()) break;
            const auto now = Clock::now();
            for (Req* r : rs) {
                r->status = SERVE_RUNNING;
                r->t_start = now;
                r->batched = 1;
            }
            running_ += static_cast<int>(rs.size());
            if (running_ > peak_running_) peak_running_ = running_;
            ++batches_;
            batched_ += static_cast<long long>(rs.size());
        }
        run_batch(rs, s);
        cv_.notify_all();
    }
    if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
}

// Bookkeeping of a request that left the device (caller holds mu_): counters,
// its transient bytes back to the budget.
void Server::finish(Req* r) {
    --running_;
    r->t_done = Clock::now();
    used_ -= r->transient;
    if (r->status == SERVE_DONE) ++done_;
    else ++failed_;
    if (r->cache_hit) ++hits_;
}

// One shared batch.  Per request: A (cached, borrowed or copied), its
// binary32 factors, B, X, R and the binary32 correction on the device; then
// batch_solve for all of them; then X back to the host and the cache.
void Server::run_batch(std::vector<Req*>& rs, cudaStream_t s) {
    const int nb = static_cast<int>(rs.size());
    if (cfg_.dry_run) {
        double n3 = 0.0;
        for (Req* r : rs) n3 += static_cast<double>(r->n) * r->n * r->n;
        std::this_thread::sleep_for(std::chrono::duration<double>(1.5e-10 * n3 + 1e-4));
        std::lock_guard<std::mutex> lk(mu_);
        for (Req* r : rs) {
            const bool fail = (r->flags & SERVE_FLAG_FAIL) != 0;
            r->status = fail ? SERVE_FAILED : SERVE_DONE;
            r->error = fail ? LU_ELAUNCH : 0;
            r->res.eta = -1.0;
            r->res.path = -1;
            r->res.precision = LU_PREC_F32;
            if (r->cache_hit) {
                Entry& e = cache_[r->matrix_id];
                e.pins -= 1;
                e.last_use = ++clock_;
            } else if (!fail && r->matrix_id != 0 && cache_.find(r->matrix_id) == cache_.end()) {
                Entry e;
                e.id = r->matrix_id;
                e.n = r->n;
                e.bytes = r->persistent;
                e.last_use = ++clock_;
                e.batched = true;
                cache_.emplace(e.id, e);
            } else {
                used_ -= r->persistent;
            }
            finish(r);
        }
        return;
    }
    struct Dev {
        double *A64 = nullptr, *B64 = nullptr, *X64 = nullptr, *R64 = nullptr, *cw = nullptr;
        float *F = nullptr, *r32 = nullptr;
        int* piv = nullptr;
        const double* Ause = nullptr;
        int ldu = 0;
        Entry* hit = nullptr;
    };
    std::vector<Dev> d(nb);
    std::vector<BatchReq> q(nb);
    std::vector<double> tol(nb);
    std::vector<int> ok(nb, 1);
    for (int i = 0; i < nb; ++i) {
        Req* r = rs[i];
        Dev& v = d[i];
        const int n = r->n, nr = r->nrhs;
        const size_t nn = static_cast<size_t>(n) * n, vs = static_cast<size_t>(n) * nr;
        const cudaMemcpyKind kin = r->dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (r->cache_hit) {
            std::lock_guard<std::mutex> lk(mu_);
            v.hit = &cache_.find(r->matrix_id)->second;
            v.A64 = v.hit->A64;
            v.F = v.hit->fac.A32;
            v.piv = v.hit->fac.piv;
            v.Ause = v.A64;
            v.ldu = n;
        }
        bool good = true;
        if (!v.hit) {
            if (r->borrow && r->dev_in) {
                v.Ause = r->bA;
                v.ldu = r->blda;
            } else {
                good = lu_malloc_async(reinterpret_cast<void**>(&v.A64), nn * sizeof(double), s) == cudaSuccess &&
                       (r->borrow ? cudaMemcpy2DAsync(v.A64, sizeof(double) * n, r->bA, sizeof(double) * r->blda,
                                                      sizeof(double) * n, n, kin, s)
                                  : cudaMemcpyAsync(v.A64, r->A.data(), nn * sizeof(double), cudaMemcpyHostToDevice,
                                                    s)) == cudaSuccess;
                v.Ause = v.A64;
                v.ldu = n;
            }
            good = good && lu_malloc_async(reinterpret_cast<void**>(&v.F), nn * sizeof(float), s) == cudaSuccess &&
                   lu_malloc_async(reinterpret_cast<void**>(&v.piv), (static_cast<size_t>(n) + 1) * sizeof(int), s) ==
                       cudaSuccess;
        }
        good = good && lu_malloc_async(reinterpret_cast<void**>(&v.B64), vs * sizeof(double), s) == cudaSuccess &&
               lu_malloc_async(reinterpret_cast<void**>(&v.X64), vs * sizeof(double), s) == cudaSuccess &&
               lu_malloc_async(reinterpret_cast<void**>(&v.R64), vs * sizeof(double), s) == cudaSuccess &&
               lu_malloc_async(reinterpret_cast<void**>(&v.r32), vs * sizeof(float), s) == cudaSuccess &&
               lu_malloc_async(reinterpret_cast<void**>(&v.cw), 2 * static_cast<size_t>(nr) * sizeof(double), s) ==
                   cudaSuccess;
        good = good && (r->borrow ? cudaMemcpy2DAsync(v.B64, sizeof(double) * nr, r->bB, sizeof(double) * r->bldb,
                                                      sizeof(double) * nr, n, kin, s)
                                  : cudaMemcpyAsync(v.B64, r->B.data(), vs * sizeof(double), cudaMemcpyHostToDevice,
                                                    s)) == cudaSuccess;
        if (!good) {
            cudaGetLastError();
            ok[i] = 0;
            r->error = LU_ENOMEM;
        }
        BatchReq& b = q[i];
        b = BatchReq{};
        b.A = v.Ause;
        b.lda = v.ldu;
        b.B = v.B64;
        b.ldb = nr;
        b.X = v.X64;
        b.R = v.R64;
        b.r = v.r32;
        b.F = v.F;
        b.piv = v.piv;
        b.cw = v.cw;
        b.n = n;
        b.nrhs = nr;
        b.factor = v.hit ? 0 : 1;
        tol[i] = r->tol;
    }
    // the requests whose buffers are in place go through the shared launches
    std::vector<BatchReq> live;
    std::vector<double> ltol;
    std::vector<int> idx_of;
    for (int i = 0; i < nb; ++i)
        if (ok[i]) {
            live.push_back(q[i]);
            ltol.push_back(tol[i]);
            idx_of.push_back(i);
        }
    std::vector<int> out, iters;
    std::vector<double> eta;
    int rc = batch_solve(live, ltol, 30, out, iters, eta, s);
    std::vector<int> code(nb, -1);                    // -1: buffers failed; 0 done; 1 singular; 2 hand over
    for (size_t j = 0; j < idx_of.size(); ++j) code[idx_of[j]] = rc ? -1 : out[j];
    for (size_t j = 0; j < idx_of.size(); ++j) {
        Req* r = rs[idx_of[j]];
        r->res = ir_result{};
        r->res.iters = iters.empty() ? 0 : iters[j];
        r->res.eta = eta.empty() ? 0.0 : eta[j];
        r->res.path = code[idx_of[j]] == 0 ? 0 : -1;
        r->res.precision = LU_PREC_F32;
        r->res.info = code[idx_of[j]] == 1 ? 1 : 0;
        if (rc) r->error = rc;
        if (code[idx_of[j]] == 0) {
            r->X.resize(static_cast<size_t>(r->n) * r->nrhs);
            if (cudaMemcpyAsync(r->X.data(), d[idx_of[j]].X64, sizeof(double) * r->X.size(), cudaMemcpyDeviceToHost,
                                s) != cudaSuccess) {
                cudaGetLastError();
                code[idx_of[j]] = -1;
                r->error = LU_ELAUNCH;
            }
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        for (int i = 0; i < nb; ++i)
            if (code[i] == 0) {
                code[i] = -1;
                rs[i]->error = LU_ELAUNCH;
            }
    }
    std::lock_guard<std::mutex> lk(mu_);
    for (int i = 0; i < nb; ++i) {
        Req* r = rs[i];
        Dev& v = d[i];
        if (v.B64) cudaFreeAsync(v.B64, s);
        if (v.X64) cudaFreeAsync(v.X64, s);
        if (v.R64) cudaFreeAsync(v.R64, s);
        if (v.r32) cudaFreeAsync(v.r32, s);
        if (v.cw) cudaFreeAsync(v.cw, s);
        if (v.hit) {
            v.hit->pins -= 1;
            v.hit->last_use = ++clock_;
        } else {
            bool keep = code[i] == 0 && r->matrix_id != 0 && cache_.find(r->matrix_id) == cache_.end();
            if (keep && v.A64 == nullptr) {
                // a borrowed device matrix: the cache keeps its own copy
                const size_t nn = static_cast<size_t>(r->n) * r->n;
                if (lu_malloc_async(reinterpret_cast<void**>(&v.A64), nn * sizeof(double), s) != cudaSuccess ||
                    cudaMemcpy2DAsync(v.A64, sizeof(double) * r->n, v.Ause, sizeof(double) * v.ldu,
                                      sizeof(double) * r->n, r->n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                    cudaGetLastError();
                    if (v.A64) cudaFreeAsync(v.A64, s);
                    v.A64 = nullptr;
                    keep = false;
                }
            }
            if (keep) {
                Entry e;
                e.id = r->matrix_id;
                e.n = r->n;
                e.A64 = v.A64;
                e.fac.n = r->n;
                e.fac.A32 = v.F;
                e.fac.piv = v.piv;
                e.fac.precision = LU_PREC_F32;
                e.bytes = r->persistent;
                e.last_use = ++clock_;
                e.batched = true;
                cache_.emplace(e.id, e);
            } else {
                if (v.A64) cudaFreeAsync(v.A64, s);
                if (v.F) cudaFreeAsync(v.F, s);
                if (v.piv) cudaFreeAsync(v.piv, s);
                used_ -= r->persistent;
            }
        }
        if (code[i] == 2) {
            // refinement on binary32 factors stopped contracting: the request
            // goes to a slot worker (the precision ladder), charged at the
            // slot path's size
            --running_;
            used_ -= r->transient;
            r->no_batch = true;
            r->batched = 0;
            r->cache_hit = 0;
            r->persistent = persistent_bytes(r->n, false);
            r->transient = transient_bytes(r->n, r->nrhs, false);
            r->status = SERVE_PENDING;
            if (r->persistent + r->transient > cfg_.hbm_budget_bytes) {
                r->status = SERVE_FAILED;
                r->error = LU_EBUSY;
                ++running_;
                used_ += r->transient;
                finish(r);
            } else {
                queue_.push_front(r);
                ++queued_[0];
            }
            continue;
        }
        r->status = code[i] == 0 ? SERVE_DONE : SERVE_FAILED;
        if (code[i] == 1) r->error = LU_EUNSUPPORTED;
        else if (code[i] < 0 && r->error == 0) r->error = LU_ELAUNCH;
        finish(r);
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
            if (lu_malloc_async(reinterpret_cast<void**>(&A64), nn * sizeof(double), s) != cudaSuccess) rc = LU_ENOMEM;
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
    if (!rc && (lu_malloc_async(reinterpret_cast<void**>(&B64), sizeof(double) * n * nr, s) != cudaSuccess ||
                lu_malloc_async(reinterpret_cast<void**>(&X64), sizeof(double) * n * nr, s) != cudaSuccess))
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
        if (lu_malloc_async(reinterpret_cast<void**>(&A64), nn * sizeof(double), s) != cudaSuccess ||
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
    st->batched = r->batched;
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
    out->batches = batches_;
    out->batched = batched_;
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
    if (cfg->batch_n_max < -1 || cfg->batch_n_max > 1024 || cfg->batch_max < 0) return -1;
    for (int r : cfg->reserved)
        if (r != 0) return -1;
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
