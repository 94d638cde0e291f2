// Batched processing of many independent plans (streams of different channel
// counts, tap counts and chunk lengths) in one call. Host side only: every
// member chunk runs the same kernels as fengine_process_chunk; the batch
// spreads the members over a pool of CUDA streams (longest work first onto
// the least-loaded stream) so small members fill the SMs that large ones
// leave idle, and joins them back into the caller's stream. The whole call
// is capturable into a CUDA graph by the caller.
#include <algorithm>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fengine.h"

struct fengine_batch_s {
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
};

namespace {

void batch_release(fengine_batch_s *b) {
    if (!b) return;
    for (cudaEvent_t e : b->done) cudaEventDestroy(e);
    for (cudaStream_t s : b->pool) cudaStreamDestroy(s);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

}  // namespace

extern "C" {

fengine_status fengine_batch_create(int32_t n_pool, fengine_batch_t *out) {
    if (!out || n_pool < 1 || n_pool > 64) return FENGINE_EINVAL;
    *out = nullptr;
    fengine_batch_s *b = new (std::nothrow) fengine_batch_s();
    if (!b) return FENGINE_ENOMEM;
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int i = 0; i < n_pool && e == cudaSuccess; i++) {
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) break;
        b->pool.push_back(s);
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) break;
        b->done.push_back(ev);
    }
    if (e != cudaSuccess) {
        batch_release(b);
        return FENGINE_ECUDA;
    }
    *out = b;
    return FENGINE_OK;
}

fengine_status fengine_batch_destroy(fengine_batch_t b) {
    if (!b) return FENGINE_EINVAL;
    for (cudaStream_t s : b->pool) cudaStreamSynchronize(s);
    batch_release(b);
    return FENGINE_OK;
}

fengine_status fengine_batch_process(fengine_batch_t b, void *cuda_stream, const fengine_chunk_desc *chunks,
                                     int32_t n, int64_t *first_spectra) {
    if (!b || (!chunks && n > 0) || n < 0) return FENGINE_EINVAL;
    if (n == 0) return FENGINE_OK;
    // members must be distinct plans (a plan's chunks are ordered through its history)
    std::vector<int> order(n);
    std::vector<double> cost(n);
    for (int i = 0; i < n; i++) {
        order[i] = i;
        fengine_info info;
        if (!chunks[i].plan || fengine_get_info(chunks[i].plan, &info) != FENGINE_OK) return FENGINE_EINVAL;
        for (int j = 0; j < i; j++)
            if (chunks[j].plan == chunks[i].plan) return FENGINE_EINVAL;
        // work ~ samples x (taps + FFT depth); channel counts and taps differ per member
        int lg = 0;
        while ((1 << lg) < 2 * info.n_channels) lg++;
        cost[i] = (double)info.n_antennas * 2.0 * (double)info.spectra_per_chunk * 2.0 * info.n_channels *
                  (double)(info.n_taps + 2 * lg + 8);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    const int np = (int)b->pool.size();
    std::vector<double> load(np, 0.0);
    std::vector<char> used(np, 0);
    if (cudaEventRecord(b->fork, st) != cudaSuccess) return FENGINE_ECUDA;
    fengine_status result = FENGINE_OK;
    for (int k = 0; k < n; k++) {
        const int i = order[k];
        const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        if (!used[s]) {
            if (cudaStreamWaitEvent(b->pool[s], b->fork, 0) != cudaSuccess) return FENGINE_ECUDA;
            used[s] = 1;
        }
        int64_t fs = 0;
        const fengine_status r =
            fengine_process_chunk(chunks[i].plan, (void *)b->pool[s], chunks[i].d_packed, chunks[i].first_sample,
                                  chunks[i].d_valid, chunks[i].d_out, chunks[i].d_heap_flags, nullptr, nullptr, &fs);
        if (r != FENGINE_OK) {
            result = r;   // members enqueued so far still run; the join below covers them
            break;
        }
        if (first_spectra) first_spectra[i] = fs;
        load[s] += cost[i];
    }
    for (int s = 0; s < np; s++) {
        if (!used[s]) continue;
        if (cudaEventRecord(b->done[s], b->pool[s]) != cudaSuccess ||
            cudaStreamWaitEvent(st, b->done[s], 0) != cudaSuccess)
            return FENGINE_ECUDA;
    }
    return result;
}

}  // extern "C"
