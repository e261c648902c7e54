// Request server: continuous batching of FP8 GEMM requests (fp8_server_*).
//
// The scheduler core (queues, admission against a workspace pool, batch
// formation, completion, statistics) is independent of the GPU; it drives an
// Executor.  CudaExecutor runs batches with the library's grouped kernels on
// one stream per tenant; SimExecutor keeps a simulated clock on the host and
// can inject launch failures (used by tests without a GPU and for capacity
// planning).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gb300fp8.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kAlign = 256;

size_t align_up(size_t v)
{
    return (v + kAlign - 1) / kAlign * kAlign;
}

struct Weight {
    int64_t N = 0, K = 0, ldw = 0;
    const uint8_t* W = nullptr;
    const uint8_t* meta = nullptr;
    const float* scale = nullptr;
    int mode = 0;
    int format = FP8_E4M3;      // fp8_format of the weight codes
};

struct Req {
    uint64_t ticket = 0;
    fp8_request r{};
    Weight w;
    size_t ws_off = 0, ws_bytes = 0;
    int status = FP8_PENDING;
    int batch_size = 0;
    double t_submit = 0, t_launch = 0, t_start = 0, t_end = 0;
};

// workspace of a request: codes [M, ldq] then scales [M]
int64_t ldq_of(const Req* q)
{
    return (q->w.K + 15) / 16 * 16;
}

size_t workspace_bytes(int64_t M, int64_t K)
{
    return align_up(static_cast<size_t>(M) * static_cast<size_t>((K + 15) / 16 * 16)) +
           align_up(static_cast<size_t>(M) * sizeof(float));
}

// First-fit allocator over [0, capacity) with coalescing of free ranges.
class Pool {
public:
    void reset(size_t capacity)
    {
        cap_ = capacity;
        free_.clear();
        if (capacity)
            free_[0] = capacity;
        in_use_ = high_ = 0;
    }
    bool alloc(size_t bytes, size_t* off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest)
                    free_[start] = rest;
                in_use_ += bytes;
                high_ = std::max(high_, in_use_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        in_use_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t capacity() const { return cap_; }
    size_t in_use() const { return in_use_; }
    size_t high_water() const { return high_; }

private:
    std::map<size_t, size_t> free_;
    size_t cap_ = 0, in_use_ = 0, high_ = 0;
};

// ------------------------------------------------------------------ executors

class Executor {
public:
    virtual ~Executor() = default;
    // Prepare streams and the pool; returns the pool capacity in *pool.
    virtual int init(const fp8_server_config& cfg, size_t* pool) = 0;
    // Enqueue the batch on the tenant's stream; *launches = kernel launches.
    virtual int launch(int tenant, const std::vector<Req*>& batch, bool batched, int max_ctas,
                       double now_us, void** handle, int* launches) = 0;
    // FP8_OK (finished; *t_start_us and *t_end_us set: the batch's stream
    // reached it, and its last kernel ended), FP8_PENDING, or the batch's error.
    virtual int query(void* handle, double now_us, double* t_start_us, double* t_end_us) = 0;
    virtual void release(void* handle) = 0;
    virtual void shutdown() = 0;
    // Called first on the scheduler thread.
    virtual void thread_init() {}
};

double gflop(const Req* q)
{
    return 2.0 * static_cast<double>(q->r.M) * q->w.N * q->w.K * 1e-9;
}

class SimExecutor : public Executor {
public:
    SimExecutor(double launch_us, double us_per_gflop, int fail_every)
        : launch_us_(launch_us), us_per_gflop_(us_per_gflop), fail_every_(fail_every) {}
    int init(const fp8_server_config& cfg, size_t* pool) override
    {
        *pool = cfg.pool_bytes ? cfg.pool_bytes : (size_t(1) << 30);
        busy_.assign(FP8_SERVER_MAX_TENANTS, 0.0);
        return FP8_OK;
    }
    int launch(int tenant, const std::vector<Req*>& batch, bool batched, int, double now_us,
               void** handle, int* launches) override
    {
        ++count_;
        double work = 0;
        for (const Req* q : batch)
            work += gflop(q);
        const double cost = launch_us_ * (batched ? 1.0 : double(batch.size())) + us_per_gflop_ * work;
        auto* b = new SimBatch;
        b->start = std::max(now_us, busy_[tenant]);
        b->end = b->start + cost;
        b->status = (fail_every_ > 0 && count_ % fail_every_ == 0) ? FP8_ERR_CUDA : FP8_OK;
        busy_[tenant] = b->end;
        *handle = b;
        *launches = batched ? 2 : 2 * static_cast<int>(batch.size());
        return FP8_OK;
    }
    int query(void* handle, double now_us, double* t_start_us, double* t_end_us) override
    {
        auto* b = static_cast<SimBatch*>(handle);
        if (now_us < b->end)
            return FP8_PENDING;
        *t_start_us = b->start;
        *t_end_us = b->end;
        return b->status;
    }
    void release(void* handle) override { delete static_cast<SimBatch*>(handle); }
    void shutdown() override {}

private:
    struct SimBatch {
        double start, end;
        int status;
    };
    double launch_us_, us_per_gflop_;
    int fail_every_;
    uint64_t count_ = 0;
    std::vector<double> busy_;
};

class CudaExecutor : public Executor {
public:
    int init(const fp8_server_config& cfg, size_t* pool) override
    {
        if (cudaGetDevice(&device_) != cudaSuccess)
            return FP8_ERR_UNSUPPORTED;
        int lo = 0, hi = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess)
            return FP8_ERR_CUDA;
        streams_.assign(cfg.num_tenants, nullptr);
        for (int t = 0; t < cfg.num_tenants; ++t) {
            const int prio = (t == cfg.latency_tenant) ? hi : lo;
            if (cudaStreamCreateWithPriority(&streams_[t], cudaStreamNonBlocking, prio) != cudaSuccess)
                return FP8_ERR_CUDA;
        }
        size_t bytes = cfg.pool_bytes;
        if (bytes == 0) {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess)
                return FP8_ERR_CUDA;
            const size_t reserve = cfg.reserve_bytes ? cfg.reserve_bytes : (size_t(1) << 30);
            if (free_b <= reserve)
                return FP8_ERR_OOM;
            bytes = (free_b - reserve) / kAlign * kAlign;
        }
        if (cudaMalloc(&pool_, bytes) != cudaSuccess)
            return FP8_ERR_OOM;
        *pool = bytes;
        if (cudaEventCreate(&epoch_) != cudaSuccess)
            return FP8_ERR_CUDA;
        return FP8_OK;
    }

    // Marks the GPU clock origin; host time of the origin is returned.
    void set_epoch(double* host_us, const std::function<double()>& now)
    {
        cudaEventRecord(epoch_, streams_[0]);
        while (cudaEventQuery(epoch_) == cudaErrorNotReady) {
        }
        *host_us = now();
    }

    int launch(int tenant, const std::vector<Req*>& batch, bool batched, int max_ctas, double,
               void** handle, int* launches) override
    {
        cudaStream_t st = streams_[tenant];
        fp8_stream_t fst = reinterpret_cast<fp8_stream_t>(st);
        int rc = FP8_OK;
        *launches = 0;
        // the start event completes when the stream reaches the batch
        cudaEvent_t ev0 = take_event();
        if (!ev0)
            return FP8_ERR_CUDA;
        if (cudaEventRecord(ev0, st) != cudaSuccess) {
            events_.push_back(ev0);
            return FP8_ERR_CUDA;
        }
        if (batched) {
            std::vector<fp8_quant_job> jobs(batch.size());
            std::vector<fp8_gemm_problem> probs(batch.size());
            for (size_t i = 0; i < batch.size(); ++i) {
                jobs[i] = quant_job(batch[i]);
                probs[i] = problem(batch[i]);
            }
            rc = fp8_quantize_e4m3_rows_grouped(jobs.data(), static_cast<int>(jobs.size()), fst);
            if (rc == FP8_OK)
                rc = gemm_fp8_grouped_ex(probs.data(), static_cast<int>(probs.size()), max_ctas, fst);
            *launches = 2;
        } else {
            for (Req* q : batch) {
                const fp8_quant_job j = quant_job(q);
                rc = fp8_quantize_e4m3(j.x, j.rows, j.cols, j.ldx, 1, j.q, j.ldq, j.dequant_scale, fst);
                if (rc != FP8_OK)
                    break;
                const fp8_gemm_problem p = problem(q);
                if (p.A_meta)
                    rc = gemm_fp8_sparse24_fmt(p.M, p.N, p.K, p.A, p.A_meta, p.B, p.ldb, p.a_scale,
                                               p.a_mode, p.b_scale, p.b_mode, p.alpha, p.C, p.ldc,
                                               p.out_dtype, p.out_transposed, p.a_format, p.b_format,
                                               fst);
                else
                    rc = gemm_fp8_dense_fmt(p.M, p.N, p.K, p.A, p.lda, p.B, p.ldb, p.a_scale, p.a_mode,
                                            p.b_scale, p.b_mode, p.alpha, p.C, p.ldc, p.out_dtype,
                                            p.a_format, p.b_format, fst);
                if (rc != FP8_OK)
                    break;
                *launches += 2;
            }
        }
        cudaEvent_t ev1 = rc == FP8_OK ? take_event() : nullptr;
        if (rc == FP8_OK && (!ev1 || cudaEventRecord(ev1, st) != cudaSuccess))
            rc = FP8_ERR_CUDA;
        if (rc != FP8_OK) {
            // kernels of this batch already enqueued may still use the
            // requests' workspace, which the caller releases on failure
            cudaStreamSynchronize(st);
            events_.push_back(ev0);
            if (ev1)
                events_.push_back(ev1);
            return rc;
        }
        *handle = new EventPair{ev0, ev1};
        return FP8_OK;
    }

    int query(void* handle, double, double* t_start_us, double* t_end_us) override
    {
        const EventPair* b = static_cast<const EventPair*>(handle);
        cudaError_t e = cudaEventQuery(b->end);
        if (e == cudaErrorNotReady)
            return FP8_PENDING;
        if (e != cudaSuccess)
            return FP8_ERR_CUDA;
        float ms0 = 0, ms1 = 0;
        if (cudaEventElapsedTime(&ms0, epoch_, b->start) != cudaSuccess ||
            cudaEventElapsedTime(&ms1, epoch_, b->end) != cudaSuccess)
            return FP8_ERR_CUDA;
        *t_start_us = epoch_host_us + 1e3 * static_cast<double>(ms0);
        *t_end_us = epoch_host_us + 1e3 * static_cast<double>(ms1);
        return FP8_OK;
    }

    void release(void* handle) override
    {
        EventPair* b = static_cast<EventPair*>(handle);
        events_.push_back(b->start);
        events_.push_back(b->end);
        delete b;
    }

    void thread_init() override { cudaSetDevice(device_); }

    void shutdown() override
    {
        for (cudaStream_t s : streams_)
            if (s)
                cudaStreamSynchronize(s);
        for (cudaEvent_t e : events_)
            cudaEventDestroy(e);
        events_.clear();
        if (epoch_)
            cudaEventDestroy(epoch_);
        epoch_ = nullptr;
        for (cudaStream_t s : streams_)
            if (s)
                cudaStreamDestroy(s);
        streams_.clear();
        if (pool_)
            cudaFree(pool_);
        pool_ = nullptr;
    }

    uint8_t* pool_base() const { return static_cast<uint8_t*>(pool_); }
    double epoch_host_us = 0;

private:
    fp8_quant_job quant_job(const Req* q) const
    {
        uint8_t* base = pool_base() + q->ws_off;
        const int64_t ldq = ldq_of(q);
        fp8_quant_job j{};
        j.x = q->r.x;
        j.rows = q->r.M;
        j.cols = q->w.K;
        j.ldx = q->r.ldx;
        j.q = base;
        j.ldq = ldq;
        j.dequant_scale = reinterpret_cast<float*>(base + align_up(size_t(q->r.M) * size_t(ldq)));
        return j;
    }

    fp8_gemm_problem problem(const Req* q) const
    {
        const fp8_quant_job j = quant_job(q);
        fp8_gemm_problem p{};
        p.K = q->w.K;
        p.alpha = q->r.alpha;
        p.C = q->r.out;
        p.ldc = q->r.ldo;
        p.out_dtype = q->r.out_dtype;
        if (q->w.meta) {
            // sparse weight on the MMA M side: out^T = W X^T, stored transposed
            p.M = q->w.N, p.N = q->r.M;
            p.A = q->w.W, p.A_meta = q->w.meta, p.lda = q->w.K / 2;
            p.a_scale = q->w.scale, p.a_mode = q->w.mode;
            p.B = j.q, p.ldb = j.ldq, p.b_scale = j.dequant_scale, p.b_mode = 1;
            p.a_format = q->w.format, p.b_format = FP8_E4M3;
            p.out_transposed = 1;
        } else {
            p.M = q->r.M, p.N = q->w.N;
            p.A = j.q, p.A_meta = nullptr, p.lda = j.ldq;
            p.a_scale = j.dequant_scale, p.a_mode = 1;
            p.B = q->w.W, p.ldb = q->w.ldw, p.b_scale = q->w.scale, p.b_mode = q->w.mode;
            p.a_format = FP8_E4M3, p.b_format = q->w.format;
            p.out_transposed = 0;
        }
        return p;
    }

    struct EventPair {
        cudaEvent_t start, end;
    };

    cudaEvent_t take_event()
    {
        if (!events_.empty()) {
            cudaEvent_t e = events_.back();
            events_.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess)
            return nullptr;
        return e;
    }

    int device_ = 0;
    std::vector<cudaStream_t> streams_;
    std::vector<cudaEvent_t> events_;
    void* pool_ = nullptr;
    cudaEvent_t epoch_ = nullptr;
};

}  // namespace

// ------------------------------------------------------------------ scheduler core

struct fp8_server {
    fp8_server_config cfg{};
    std::unique_ptr<Executor> exec;
    CudaExecutor* cuda = nullptr;           // exec when it runs on the GPU
    Clock::time_point t0;
    Pool pool;
    std::vector<Weight> weights;

    std::mutex mu;
    std::condition_variable done_cv;
    std::deque<Req*> queue[FP8_SERVER_MAX_TENANTS];
    std::unordered_map<uint64_t, Req*> reqs;
    uint64_t next_ticket = 1;
    bool stopping = false;
    fp8_server_stats stats{};

    struct Batch {
        void* handle;
        std::vector<Req*> reqs;
    };
    std::deque<Batch> inflight[FP8_SERVER_MAX_TENANTS];
    std::thread sched;

    double now_us() const
    {
        return std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
    }

    // A batch formed under the lock and enqueued on the GPU without it.
    struct Formed {
        int tenant;
        int max_ctas;
        std::vector<Req*> reqs;
        void* handle = nullptr;
        int launches = 0;
        int rc = FP8_OK;
        double t_launch = 0;
    };

    // Scheduler thread: retire finished batches, form new ones under the
    // lock, enqueue them with the lock released (so submit, poll and wait
    // never wait on a launch), then record them.  It spins (yielding) while
    // work is around and backs off to short sleeps after ~2 ms without any.
    void run()
    {
        exec->thread_init();
        double last_progress = now_us();
        std::vector<Formed> todo;
        for (;;) {
            bool progress = false;
            todo.clear();
            {
                std::unique_lock<std::mutex> lk(mu);
                progress |= retire_locked();
                if (stopping && idle_locked())
                    break;
                if (!stopping)
                    form_locked(&todo);
            }
            for (Formed& b : todo) {
                b.t_launch = now_us();
                b.rc = exec->launch(b.tenant, b.reqs, cfg.batching != 0, b.max_ctas, b.t_launch, &b.handle,
                                    &b.launches);
            }
            if (!todo.empty()) {
                std::unique_lock<std::mutex> lk(mu);
                record_locked(&todo);
                progress = true;
            }
            const double now = now_us();
            if (progress)
                last_progress = now;
            else if (now - last_progress > 2000.0)
                std::this_thread::sleep_for(std::chrono::microseconds(50));
            else
                std::this_thread::yield();
        }
    }

    bool idle_locked()
    {
        for (int t = 0; t < cfg.num_tenants; ++t)
            if (!inflight[t].empty())
                return false;
        return true;
    }

    bool retire_locked()
    {
        bool any = false;
        const double now = now_us();
        for (int t = 0; t < cfg.num_tenants; ++t) {
            while (!inflight[t].empty()) {
                Batch& b = inflight[t].front();
                double t_start = now, t_end = now;
                const int rc = exec->query(b.handle, now, &t_start, &t_end);
                if (rc == FP8_PENDING)
                    break;
                for (Req* q : b.reqs) {
                    q->status = rc;
                    q->t_start = t_start;
                    q->t_end = t_end;
                    pool.release(q->ws_off, q->ws_bytes);
                    if (rc == FP8_OK)
                        ++stats.completed;
                    else
                        ++stats.failed;
                }
                exec->release(b.handle);
                inflight[t].pop_front();
                any = true;
            }
        }
        if (any)
            done_cv.notify_all();
        return any;
    }

    // Take queued requests into batches (FIFO per tenant, admitted while
    // their workspace fits the pool).  The latency tenant first, with no
    // in-flight limit and batches of at most latency_max_batch; the bulk
    // tenants in index order, each while it has an in-flight slot.
    void form_locked(std::vector<Formed>* out)
    {
        int formed[FP8_SERVER_MAX_TENANTS] = {};
        for (int k = -1; k < cfg.num_tenants; ++k) {
            const int t = (k < 0) ? cfg.latency_tenant : k;
            if (t < 0 || (k >= 0 && t == cfg.latency_tenant))
                continue;
            const bool latency = t == cfg.latency_tenant;
            const int cap = !cfg.batching ? 1 : (latency ? cfg.latency_max_batch : cfg.max_batch);
            while (!queue[t].empty() &&
                   (!cfg.batching || latency ||
                    static_cast<int>(inflight[t].size()) + formed[t] < cfg.max_inflight)) {
                Formed b;
                b.tenant = t;
                b.max_ctas = latency ? cfg.latency_max_ctas : cfg.bulk_max_ctas;
                while (!queue[t].empty() && static_cast<int>(b.reqs.size()) < cap) {
                    Req* q = queue[t].front();
                    // bulk tenants leave latency_pool_bytes of the pool to the
                    // latency tenant, so a full pool never holds its requests
                    if (!latency && pool.in_use() + q->ws_bytes + cfg.latency_pool_bytes > pool.capacity())
                        break;
                    if (!pool.alloc(q->ws_bytes, &q->ws_off))
                        break;                      // FIFO: wait for space
                    b.reqs.push_back(q);
                    queue[t].pop_front();
                }
                if (b.reqs.empty())
                    break;
                ++formed[t];
                out->push_back(std::move(b));
            }
        }
    }

    void record_locked(std::vector<Formed>* todo)
    {
        bool failed = false;
        for (Formed& b : *todo) {
            stats.kernel_launches += b.launches;
            if (b.rc != FP8_OK) {
                for (Req* q : b.reqs) {
                    q->status = b.rc;
                    q->t_launch = q->t_start = q->t_end = b.t_launch;
                    pool.release(q->ws_off, q->ws_bytes);
                    ++stats.failed;
                }
                failed = true;
                continue;
            }
            for (Req* q : b.reqs) {
                q->t_launch = b.t_launch;
                q->batch_size = static_cast<int>(b.reqs.size());
            }
            ++stats.batches;
            stats.max_batch_seen = std::max<uint64_t>(stats.max_batch_seen, b.reqs.size());
            inflight[b.tenant].push_back(Batch{b.handle, std::move(b.reqs)});
        }
        if (failed)
            done_cv.notify_all();
    }
};

namespace {

int normalise(const fp8_server_config* in, fp8_server_config* out)
{
    if (!in)
        return FP8_ERR_INVALID;
    fp8_server_config c = *in;
    if (c.num_tenants < 1 || c.num_tenants > FP8_SERVER_MAX_TENANTS)
        return FP8_ERR_INVALID;
    if (c.latency_tenant < -1 || c.latency_tenant >= c.num_tenants)
        return FP8_ERR_INVALID;
    if (c.max_batch <= 0 || c.max_batch > FP8_GROUPED_MAX_PROBLEMS)
        c.max_batch = FP8_GROUPED_MAX_PROBLEMS;
    if (c.max_batch > FP8_QUANT_GROUPED_MAX)
        c.max_batch = FP8_QUANT_GROUPED_MAX;
    if (c.max_inflight <= 0)
        c.max_inflight = 4;
    if (c.latency_max_batch <= 0)
        c.latency_max_batch = 1;
    if (c.latency_max_batch > c.max_batch)
        c.latency_max_batch = c.max_batch;
    if (c.bulk_max_ctas < 0)
        c.bulk_max_ctas = 0;
    if (c.latency_max_ctas < 0)
        c.latency_max_ctas = 0;
    if (c.latency_tenant < 0)
        c.latency_pool_bytes = 0;
    *out = c;
    return FP8_OK;
}

int start(fp8_server* s, fp8_server** out)
{
    size_t cap = 0;
    int rc = s->exec->init(s->cfg, &cap);
    if (rc != FP8_OK) {
        s->exec->shutdown();
        delete s;
        return rc;
    }
    s->pool.reset(cap);
    s->stats.pool_bytes = cap;
    s->t0 = Clock::now();
    if (s->cuda)
        s->cuda->set_epoch(&s->cuda->epoch_host_us, [s] { return s->now_us(); });
    s->sched = std::thread([s] { s->run(); });
    *out = s;
    return FP8_OK;
}

}  // namespace

extern "C" int fp8_server_create(const fp8_server_config* cfg, fp8_server** out)
{
    if (!out)
        return FP8_ERR_INVALID;
    auto* s = new fp8_server;
    int rc = normalise(cfg, &s->cfg);
    if (rc != FP8_OK) {
        delete s;
        return rc;
    }
    auto* ce = new CudaExecutor;
    s->cuda = ce;
    s->exec.reset(ce);
    return start(s, out);
}

extern "C" int fp8_server_create_simulated(const fp8_server_config* cfg, double launch_us,
                                           double us_per_gflop, int fail_every, fp8_server** out)
{
    if (!out || launch_us < 0 || us_per_gflop < 0)
        return FP8_ERR_INVALID;
    auto* s = new fp8_server;
    int rc = normalise(cfg, &s->cfg);
    if (rc != FP8_OK) {
        delete s;
        return rc;
    }
    s->exec.reset(new SimExecutor(launch_us, us_per_gflop, fail_every));
    return start(s, out);
}

extern "C" int fp8_server_destroy(fp8_server* s)
{
    if (!s)
        return FP8_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        for (int t = 0; t < s->cfg.num_tenants; ++t) {
            for (Req* q : s->queue[t]) {
                q->status = FP8_ERR_INVALID;
                ++s->stats.failed;
            }
            s->queue[t].clear();
        }
    }
    s->sched.join();
    s->exec->shutdown();
    for (auto& kv : s->reqs)
        delete kv.second;
    delete s;
    return FP8_OK;
}

extern "C" int fp8_server_register_weight(fp8_server* s, int64_t N, int64_t K, const uint8_t* W,
                                          int64_t ldw, const uint8_t* W_meta, const float* w_scale,
                                          int w_mode, uint64_t* handle)
{
    return fp8_server_register_weight_fmt(s, N, K, W, ldw, W_meta, w_scale, w_mode, FP8_E4M3, handle);
}

extern "C" int fp8_server_register_weight_fmt(fp8_server* s, int64_t N, int64_t K, const uint8_t* W,
                                              int64_t ldw, const uint8_t* W_meta, const float* w_scale,
                                              int w_mode, int w_format, uint64_t* handle)
{
    if (!s || !W || !w_scale || !handle || (w_mode != 0 && w_mode != 1) ||
        (w_format != FP8_E4M3 && w_format != FP8_E5M2))
        return FP8_ERR_INVALID;
    if (N <= 0 || K <= 0 || K % 16 != 0 || N > INT32_MAX / 2 || K > INT32_MAX / 2)
        return FP8_ERR_SHAPE;
    if (W_meta) {
        if (K % 128 != 0)
            return FP8_ERR_SHAPE;
    } else if (ldw < K || ldw % 16 != 0) {
        return FP8_ERR_SHAPE;
    }
    Weight w;
    w.N = N, w.K = K, w.ldw = W_meta ? K / 2 : ldw, w.W = W, w.meta = W_meta, w.scale = w_scale,
    w.mode = w_mode, w.format = w_format;
    std::lock_guard<std::mutex> lk(s->mu);
    s->weights.push_back(w);
    *handle = s->weights.size();                 // 1-based
    return FP8_OK;
}

extern "C" int fp8_server_submit(fp8_server* s, const fp8_request* r, uint64_t* ticket)
{
    if (!s || !r || !ticket)
        return FP8_ERR_INVALID;
    if (r->tenant < 0 || r->tenant >= s->cfg.num_tenants || r->M < 0 ||
        (r->out_dtype != 0 && r->out_dtype != 1))
        return FP8_ERR_INVALID;
    auto* q = new Req;
    q->r = *r;
    q->t_submit = s->now_us();
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->weight == 0 || r->weight > s->weights.size()) {
        delete q;
        return FP8_ERR_INVALID;
    }
    q->w = s->weights[r->weight - 1];
    if (r->M > 0 && (!r->x || !r->out || r->ldx < q->w.K || r->ldo < q->w.N)) {
        delete q;
        return r->x && r->out ? FP8_ERR_SHAPE : FP8_ERR_INVALID;
    }
    if (s->stopping) {
        delete q;
        return FP8_ERR_INVALID;
    }
    q->ws_bytes = workspace_bytes(std::max<int64_t>(r->M, 1), q->w.K);
    const size_t limit = s->pool.capacity() - (r->tenant == s->cfg.latency_tenant
                                                  ? 0 : std::min(s->cfg.latency_pool_bytes, s->pool.capacity()));
    if (q->ws_bytes > limit) {
        ++s->stats.rejected;
        delete q;
        return FP8_ERR_OOM;
    }
    q->ticket = s->next_ticket++;
    s->reqs[q->ticket] = q;
    s->queue[r->tenant].push_back(q);
    ++s->stats.submitted;
    *ticket = q->ticket;
    return FP8_OK;
}

namespace {

int collect_locked(fp8_server* s, uint64_t ticket, fp8_result* res, bool* found)
{
    auto it = s->reqs.find(ticket);
    *found = it != s->reqs.end();
    if (!*found)
        return FP8_ERR_INVALID;
    Req* q = it->second;
    if (q->status == FP8_PENDING)
        return FP8_PENDING;
    if (res) {
        res->status = q->status;
        res->batch_size = q->batch_size;
        res->t_submit_us = q->t_submit;
        res->t_launch_us = q->t_launch;
        res->t_end_us = q->t_end;
        res->t_start_us = q->t_start;
    }
    const int st = q->status;
    s->reqs.erase(it);
    delete q;
    return st;
}

}  // namespace

extern "C" int fp8_server_poll(fp8_server* s, uint64_t ticket, fp8_result* res)
{
    if (!s)
        return FP8_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    bool found = false;
    return collect_locked(s, ticket, res, &found);
}

extern "C" int fp8_server_wait(fp8_server* s, uint64_t ticket, fp8_result* res, double timeout_s)
{
    if (!s)
        return FP8_ERR_INVALID;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(std::max(0.0, timeout_s)));
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool found = false;
        const int rc = collect_locked(s, ticket, res, &found);
        if (rc != FP8_PENDING || !found)
            return rc;
        if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            const int rc2 = collect_locked(s, ticket, res, &found);
            return rc2;
        }
    }
}

extern "C" int fp8_server_get_stats(fp8_server* s, fp8_server_stats* out)
{
    if (!s || !out)
        return FP8_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->pool_bytes = s->pool.capacity();
    out->pool_in_use = s->pool.in_use();
    out->pool_high_water = s->pool.high_water();
    return FP8_OK;
}

extern "C" double fp8_server_now_us(fp8_server* s)
{
    return s ? s->now_us() : 0.0;
}
