// Streaming service: continuous batching of chunk requests from many F-engine
// plans (Sec. 3.1: the engine is a pipeline of chunks whose host-to-device
// copies, computation and device-to-host copies overlap).
//
// A request is one chunk of one plan in host memory. A dispatcher thread
// admits queued requests in arrival order as soon as (a) the device memory
// they need (input and output buffers) fits in the budget next to the
// requests in flight, and (b) a CUDA stream is free; a plan stays on one
// stream, so its chunks run in order while different plans overlap on the
// device. Each admitted request runs H2D copy -> fengine_process_chunk ->
// D2H copy on its stream; a host callback at the end of the stream work
// records its completion time and hands the memory back. Delay and gain
// updates are requests too, applied in order with the plan's chunks. All
// waits are bounded; nothing here waits on the device from device code.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fengine.h"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    int kind = 0;                      // 0 chunk, 1 delay update, 2 gain update
    fengine_plan_t plan = nullptr;
    const uint8_t *h_in = nullptr;
    int8_t *h_out = nullptr;
    const uint8_t *h_valid = nullptr;  // optional received-heap flags of the chunk
    uint8_t *h_flags = nullptr;        // optional output-heap flags
    size_t valid_bytes = 0, flag_bytes = 0;
    int64_t first_sample = 0;
    size_t in_bytes = 0, out_bytes = 0;
    // updates
    int32_t ant = 0, pol = 0;
    int64_t t_apply = 0, t_ref = 0;
    double d[4] = {0, 0, 0, 0};
    std::vector<float> gains;
    // progress
    clk::time_point t_submit, t_admit, t_done;
    int stream = -1;
    void *d_in = nullptr, *d_out = nullptr, *d_valid = nullptr, *d_flags = nullptr;
    fengine_status status = FENGINE_OK;
    bool done = false;
    bool deferred = false;
};

constexpr int kLatBinsPerOctave = 64;
constexpr int kLatBins = 40 * kLatBinsPerOctave;   // 1 us .. 2^40 us

int latency_bin(double us) {
    if (!(us >= 1.0)) return 0;
    const int b = (int)std::floor(std::log2(us) * kLatBinsPerOctave);
    return std::min(b, kLatBins - 1);
}

}  // namespace

struct fengine_service_s {
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_busy;      // requests in flight per stream
    int64_t budget = 0, in_use = 0, peak = 0;
    std::map<fengine_plan_t, int> plan_stream;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<int64_t, std::shared_ptr<Request>> all;
    // completed-request latencies as a histogram of fixed size: bin b holds
    // latencies in [2^(b/kLatBinsPerOctave), 2^((b+1)/kLatBinsPerOctave)) us
    // (1.1 % wide), so a long-lived service keeps constant memory
    std::vector<int64_t> lat_hist = std::vector<int64_t>(kLatBins, 0);
    double lat_max_us = 0.0;
    int64_t next_ticket = 1;
    int64_t admitted = 0, completed = 0, deferred = 0, failed = 0;
    std::mutex mu;
    std::condition_variable cv;        // dispatcher wake-up
    std::condition_variable done_cv;   // completions
    bool stop = false;
    std::thread worker;
    int device = 0;
};

namespace {

struct CallbackCtx {
    fengine_service_s *svc;
    std::shared_ptr<Request> req;
};

// Runs on a CUDA host-callback thread once the request's stream work is done.
// Makes no CUDA calls; the dispatcher frees the device buffers.
void CUDART_CB on_complete(void *arg) {
    CallbackCtx *ctx = static_cast<CallbackCtx *>(arg);
    {
        std::lock_guard<std::mutex> lk(ctx->svc->mu);
        ctx->req->t_done = clk::now();
        ctx->req->done = true;
    }
    ctx->svc->cv.notify_all();
    ctx->svc->done_cv.notify_all();
    delete ctx;
}

fengine_status launch_chunk(fengine_service_s *s, const std::shared_ptr<Request> &r) {
    cudaStream_t st = s->streams[r->stream];
    if (cudaMallocAsync(&r->d_in, r->in_bytes, st) != cudaSuccess) return FENGINE_ENOMEM;
    if (cudaMallocAsync(&r->d_out, r->out_bytes, st) != cudaSuccess) return FENGINE_ENOMEM;
    if (r->h_valid && cudaMallocAsync(&r->d_valid, r->valid_bytes, st) != cudaSuccess) return FENGINE_ENOMEM;
    if (r->h_flags && cudaMallocAsync(&r->d_flags, r->flag_bytes, st) != cudaSuccess) return FENGINE_ENOMEM;
    if (cudaMemcpyAsync(r->d_in, r->h_in, r->in_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FENGINE_ECUDA;
    if (r->h_valid &&
        cudaMemcpyAsync(r->d_valid, r->h_valid, r->valid_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FENGINE_ECUDA;
    const fengine_status ps =
        fengine_process_chunk(r->plan, (void *)st, (const uint8_t *)r->d_in, r->first_sample,
                              (const uint8_t *)r->d_valid, (int8_t *)r->d_out, (uint8_t *)r->d_flags, nullptr,
                              nullptr, nullptr);
    if (ps != FENGINE_OK) return ps;
    if (cudaMemcpyAsync(r->h_out, r->d_out, r->out_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return FENGINE_ECUDA;
    if (r->h_flags && cudaMemcpyAsync(r->h_flags, r->d_flags, r->flag_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return FENGINE_ECUDA;
    return FENGINE_OK;
}

void dispatcher(fengine_service_s *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // retire completed requests: give their memory and stream slot back
        bool retired = false;
        for (auto &kv : s->all) {
            Request &r = *kv.second;
            if (r.done && r.stream >= 0 && r.kind == 0 && (r.d_in || r.d_out)) {
                cudaFreeAsync(r.d_in, s->streams[r.stream]);
                cudaFreeAsync(r.d_out, s->streams[r.stream]);
                if (r.d_valid) cudaFreeAsync(r.d_valid, s->streams[r.stream]);
                if (r.d_flags) cudaFreeAsync(r.d_flags, s->streams[r.stream]);
                r.d_in = r.d_out = r.d_valid = r.d_flags = nullptr;
                s->in_use -= (int64_t)(r.in_bytes + r.out_bytes);
                s->stream_busy[r.stream]--;
                s->completed++;
                const double us = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
                s->lat_hist[latency_bin(us)]++;
                s->lat_max_us = std::max(s->lat_max_us, us);
                retired = true;
            }
        }
        if (retired) s->done_cv.notify_all();   // waiters need the buffers released too
        if (s->stop && s->queue.empty()) break;
        // admit in arrival order; a request that cannot go blocks later
        // requests of its own plan only (per-plan order), not other plans
        std::map<fengine_plan_t, bool> blocked;
        bool progressed = false;
        for (auto it = s->queue.begin(); it != s->queue.end();) {
            std::shared_ptr<Request> r = *it;
            if (blocked[r->plan]) {
                ++it;
                continue;
            }
            auto ps = s->plan_stream.find(r->plan);
            int si;
            if (ps == s->plan_stream.end()) {
                // least-busy stream for a plan seen for the first time
                si = (int)(std::min_element(s->stream_busy.begin(), s->stream_busy.end()) - s->stream_busy.begin());
                s->plan_stream[r->plan] = si;
            } else {
                si = ps->second;
            }
            if (r->kind != 0) {
                // updates touch only host state of the plan; they take effect
                // from the plan's next chunk, which is launched after them
                r->stream = si;
                r->status = r->kind == 1
                    ? fengine_set_delay(r->plan, r->ant, r->pol, r->t_apply, r->t_ref, r->d[0], r->d[1], r->d[2], r->d[3])
                    : fengine_set_gains(r->plan, r->ant, r->pol, r->gains.data(), r->t_apply);
                r->done = true;
                r->t_done = clk::now();
                it = s->queue.erase(it);
                progressed = true;
                s->done_cv.notify_all();
                continue;
            }
            const int64_t need = (int64_t)(r->in_bytes + r->out_bytes);
            if (s->in_use + need > s->budget) {
                if (!r->deferred) {
                    r->deferred = true;
                    s->deferred++;
                }
                blocked[r->plan] = true;
                if (need > s->budget) {   // can never fit
                    r->status = FENGINE_EBUSY;
                    r->done = true;
                    r->t_done = clk::now();
                    s->failed++;
                    it = s->queue.erase(it);
                    s->done_cv.notify_all();
                    continue;
                }
                ++it;
                continue;
            }
            r->stream = si;
            r->t_admit = clk::now();
            s->in_use += need;
            s->peak = std::max(s->peak, s->in_use);
            s->stream_busy[si]++;
            s->admitted++;
            it = s->queue.erase(it);
            progressed = true;
            lk.unlock();
            fengine_status st = launch_chunk(s, r);
            CallbackCtx *ctx = nullptr;
            if (st == FENGINE_OK) {
                ctx = new (std::nothrow) CallbackCtx{s, r};
                if (!ctx || cudaLaunchHostFunc(s->streams[si], on_complete, ctx) != cudaSuccess) {
                    delete ctx;
                    st = FENGINE_ECUDA;
                }
            }
            lk.lock();
            if (st != FENGINE_OK) {
                // the request failed before its completion callback was queued:
                // release what it holds once the stream passes its work
                r->status = st;
                if (r->d_in) cudaFreeAsync(r->d_in, s->streams[si]);
                if (r->d_out) cudaFreeAsync(r->d_out, s->streams[si]);
                if (r->d_valid) cudaFreeAsync(r->d_valid, s->streams[si]);
                if (r->d_flags) cudaFreeAsync(r->d_flags, s->streams[si]);
                r->d_in = r->d_out = r->d_valid = r->d_flags = nullptr;
                s->in_use -= need;
                s->stream_busy[si]--;
                s->failed++;
                r->t_done = clk::now();
                r->done = true;
                s->done_cv.notify_all();
            }
            it = s->queue.begin();    // the queue may have changed while unlocked
        }
        if (!progressed) s->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

}  // namespace

extern "C" {

fengine_status fengine_service_create(const fengine_service_config *cfg, fengine_service_t *out) {
    if (!cfg || !out || cfg->n_streams < 1 || cfg->n_streams > 64 || cfg->hbm_budget_bytes <= 0)
        return FENGINE_EINVAL;
    *out = nullptr;
    fengine_service_s *s = new (std::nothrow) fengine_service_s();
    if (!s) return FENGINE_ENOMEM;
    cudaGetDevice(&s->device);
    s->budget = cfg->hbm_budget_bytes;
    // keep up to the budget cached in the device's stream-ordered pool so
    // steady-state requests do not go back to the driver for memory
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        uint64_t thr = (uint64_t)cfg->hbm_budget_bytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    for (int i = 0; i < cfg->n_streams; i++) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return FENGINE_ECUDA;
        }
        s->streams.push_back(st);
        s->stream_busy.push_back(0);
    }
    s->worker = std::thread(dispatcher, s);
    *out = s;
    return FENGINE_OK;
}

fengine_status fengine_service_submit(fengine_service_t s, fengine_plan_t plan, const uint8_t *h_packed,
                                      int64_t first_sample, const uint8_t *h_valid, int8_t *h_out,
                                      uint8_t *h_heap_flags, int64_t *ticket) {
    if (!s || !plan || !h_packed || !h_out || !ticket) return FENGINE_EINVAL;
    fengine_info info;
    if (fengine_get_info(plan, &info) != FENGINE_OK) return FENGINE_EINVAL;
    auto r = std::make_shared<Request>();
    r->kind = 0;
    r->plan = plan;
    r->h_in = h_packed;
    r->h_out = h_out;
    r->h_valid = h_valid;
    r->h_flags = h_heap_flags;
    r->first_sample = first_sample;
    const int64_t L = info.spectra_per_chunk * 2 * info.n_channels;
    r->in_bytes = (size_t)info.n_antennas * 2 * (size_t)L / 4 * 5;
    r->out_bytes = (size_t)info.out_bytes;
    r->valid_bytes = (size_t)info.n_antennas * 2 * (size_t)(L / 4096);
    r->flag_bytes = (size_t)info.n_antennas * (size_t)info.heaps_per_chunk;
    r->t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return FENGINE_EBUSY;
        r->ticket = s->next_ticket++;
        s->all[r->ticket] = r;
        s->queue.push_back(r);
        *ticket = r->ticket;
    }
    s->cv.notify_all();
    return FENGINE_OK;
}

fengine_status fengine_service_set_delay(fengine_service_t s, fengine_plan_t plan, int32_t ant, int32_t pol,
                                         int64_t t_apply, int64_t t_ref, double delay, double delay_rate,
                                         double phase, double phase_rate) {
    if (!s || !plan) return FENGINE_EINVAL;
    auto r = std::make_shared<Request>();
    r->kind = 1;
    r->plan = plan;
    r->ant = ant;
    r->pol = pol;
    r->t_apply = t_apply;
    r->t_ref = t_ref;
    r->d[0] = delay;
    r->d[1] = delay_rate;
    r->d[2] = phase;
    r->d[3] = phase_rate;
    r->t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return FENGINE_EBUSY;
        r->ticket = s->next_ticket++;
        s->all[r->ticket] = r;
        s->queue.push_back(r);
    }
    s->cv.notify_all();
    return FENGINE_OK;
}

fengine_status fengine_service_set_gains(fengine_service_t s, fengine_plan_t plan, int32_t ant, int32_t pol,
                                         const float *gains_re_im, int64_t t_apply) {
    if (!s || !plan || !gains_re_im) return FENGINE_EINVAL;
    fengine_info info;
    if (fengine_get_info(plan, &info) != FENGINE_OK) return FENGINE_EINVAL;
    auto r = std::make_shared<Request>();
    r->kind = 2;
    r->plan = plan;
    r->ant = ant;
    r->pol = pol;
    r->gains.assign(gains_re_im, gains_re_im + 2 * (size_t)info.n_channels);
    r->t_apply = t_apply;
    r->t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return FENGINE_EBUSY;
        r->ticket = s->next_ticket++;
        s->all[r->ticket] = r;
        s->queue.push_back(r);
    }
    s->cv.notify_all();
    return FENGINE_OK;
}

fengine_status fengine_service_wait(fengine_service_t s, int64_t ticket, int32_t timeout_ms, double *latency_us) {
    if (!s) return FENGINE_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return FENGINE_EINVAL;
    std::shared_ptr<Request> r = it->second;
    auto pred = [&] { return r->done && (r->kind != 0 || (!r->d_in && !r->d_out)); };
    if (timeout_ms < 0) {
        s->done_cv.wait(lk, pred);
    } else if (!s->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
        return FENGINE_ETIMEOUT;
    }
    if (latency_us) *latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    const fengine_status st = r->status;
    s->all.erase(ticket);
    return st;
}

fengine_status fengine_service_get_stats(fengine_service_t s, fengine_service_stats *out) {
    if (!s || !out) return FENGINE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    int64_t n_lat = 0;
    for (int64_t c : s->lat_hist) n_lat += c;
    // q-quantile: the geometric centre of the bin holding the ceil(q n)-th
    // smallest latency (relative resolution 1.1 %), capped at the maximum
    auto pct = [&](double q) {
        if (n_lat == 0) return 0.0;
        const int64_t rank = std::max<int64_t>(1, (int64_t)std::ceil(q * (double)n_lat));
        int64_t acc = 0;
        for (int b = 0; b < kLatBins; ++b) {
            acc += s->lat_hist[b];
            if (acc >= rank) return std::min(s->lat_max_us, std::exp2(((double)b + 0.5) / kLatBinsPerOctave));
        }
        return s->lat_max_us;
    };
    out->admitted = s->admitted;
    out->completed = s->completed;
    out->deferred = s->deferred;
    out->failed = s->failed;
    out->queued = (int64_t)s->queue.size();
    out->bytes_in_use = s->in_use;
    out->peak_bytes = s->peak;
    out->latency_p50_us = pct(0.50);
    out->latency_p99_us = pct(0.99);
    out->latency_max_us = s->lat_max_us;
    return FENGINE_OK;
}

fengine_status fengine_service_destroy(fengine_service_t s) {
    if (!s) return FENGINE_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    // drain: the dispatcher exits once the queue is empty; then wait for the
    // work in flight (bounded by the streams' own progress)
    s->worker.join();
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    {
        std::unique_lock<std::mutex> lk(s->mu);
        for (auto &kv : s->all) {
            Request &r = *kv.second;
            if (r.stream >= 0 && (r.d_in || r.d_out)) {
                cudaFreeAsync(r.d_in, s->streams[r.stream]);
                cudaFreeAsync(r.d_out, s->streams[r.stream]);
                if (r.d_valid) cudaFreeAsync(r.d_valid, s->streams[r.stream]);
                if (r.d_flags) cudaFreeAsync(r.d_flags, s->streams[r.stream]);
                r.d_in = r.d_out = r.d_valid = r.d_flags = nullptr;
            }
        }
    }
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete s;
    return FENGINE_OK;
}

}  // extern "C"
