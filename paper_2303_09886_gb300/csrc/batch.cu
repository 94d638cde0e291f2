// Batched processing of many independent plans (streams of different channel
// counts, tap counts and chunk lengths) in one call. Every member computes
// exactly what fengine_process_chunk computes for it. Members in the FP32
// form are grouped: their small per-call kernels (delay table, lost-data
// flags, history tail) run spread over a pool of CUDA streams, and their
// phase-1 and phase-2 launches are merged into one grid per kernel
// instantiation (the members with the same taps and split), round by round
// over slabs; the other members run whole on the pool's streams meanwhile.
// Everything forks from and joins back into the caller's stream, so the
// call is capturable into a CUDA graph.
#include <algorithm>
#include <cstdint>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fengine.h"
#include "fe_internal.cuh"

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
    auto pick = [&](int i) -> int {
        const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[s] += cost[i];
        return s;
    };
    auto use = [&](int s) -> bool {
        if (!used[s]) {
            if (cudaStreamWaitEvent(b->pool[s], b->fork, 0) != cudaSuccess) return false;
            used[s] = 1;
        }
        return true;
    };
    fengine_status result = FENGINE_OK;

    // 1. the FP32 members' small kernels; their phase launches come back
    std::vector<std::unique_ptr<fe::DeferredCall>> deferred;
    std::vector<double> deferred_cost;
    std::vector<int> whole;   // members of the other forms
    for (int k = 0; k < n && result == FENGINE_OK; k++) {
        const int i = order[k];
        if (!fe::plan_defers(chunks[i].plan)) {
            whole.push_back(i);
            continue;
        }
        const int s = pick(i);
        if (!use(s)) return FENGINE_ECUDA;
        auto dc = std::make_unique<fe::DeferredCall>();
        bool was_deferred = false;
        int64_t fs = 0;
        const fengine_status r = fe::process_chunk_deferred(chunks[i].plan, b->pool[s], chunks[i].d_packed,
                                                            chunks[i].first_sample, chunks[i].d_valid, chunks[i].d_out,
                                                            chunks[i].d_heap_flags, &fs, dc.get(), &was_deferred);
        if (r != FENGINE_OK) {
            result = r;   // members enqueued so far still run; the joins below cover them
            break;
        }
        if (first_spectra) first_spectra[i] = fs;
        if (was_deferred) {
            deferred.push_back(std::move(dc));
            deferred_cost.push_back(cost[i]);
        }
    }
    // 2. everything after this point follows every member's small kernels
    for (int sidx = 0; sidx < np; sidx++) {
        if (!used[sidx]) continue;
        if (cudaEventRecord(b->done[sidx], b->pool[sidx]) != cudaSuccess ||
            cudaStreamWaitEvent(st, b->done[sidx], 0) != cudaSuccess)
            return FENGINE_ECUDA;
    }
    if (cudaEventRecord(b->fork, st) != cudaSuccess) return FENGINE_ECUDA;
    std::vector<char> forked(np, 0);
    auto use2 = [&](int sidx) -> bool {
        if (!forked[sidx]) {
            if (cudaStreamWaitEvent(b->pool[sidx], b->fork, 0) != cudaSuccess) return false;
            forked[sidx] = used[sidx] = 1;
        }
        return true;
    };
    std::fill(load.begin(), load.end(), 0.0);
    // 3. the other members whole on the pool's streams
    for (size_t k = 0; k < whole.size() && result == FENGINE_OK; k++) {
        const int i = whole[k];
        const int sidx = pick(i);
        if (!use2(sidx)) return FENGINE_ECUDA;
        int64_t fs = 0;
        const fengine_status r =
            fengine_process_chunk(chunks[i].plan, (void *)b->pool[sidx], chunks[i].d_packed, chunks[i].first_sample,
                                  chunks[i].d_valid, chunks[i].d_out, chunks[i].d_heap_flags, nullptr, nullptr, &fs);
        if (r != FENGINE_OK) {
            result = r;
            break;
        }
        if (first_spectra) first_spectra[i] = fs;
    }
    // 4. the FP32 members in groups of one kernel instantiation each (taps, N1,
    // N2): per group, slab round by slab round, one phase-1 grid then one
    // phase-2 grid, the group's chain on one pool stream (groups overlap)
    std::map<std::tuple<int, int, int>, std::vector<const fe::DeferredCall *>> groups;
    std::map<std::tuple<int, int, int>, double> gcost;
    for (size_t k = 0; k < deferred.size(); k++) {
        const auto key = std::make_tuple(deferred[k]->T, deferred[k]->N1, deferred[k]->N2);
        groups[key].push_back(deferred[k].get());
        gcost[key] += deferred_cost[k];
    }
    std::vector<std::pair<double, std::tuple<int, int, int>>> gorder;
    for (auto &kv : groups) gorder.emplace_back(gcost[kv.first], kv.first);
    std::stable_sort(gorder.begin(), gorder.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
    auto grouped = std::make_unique<fe::Phase1Group>();
    auto grouped2 = std::make_unique<fe::Phase2Group>();
    const int wave = fe::phase2w_wave();
    for (const auto &go : gorder) {
        const auto &v = groups[go.second];
        const int T = std::get<0>(go.second), N1 = std::get<1>(go.second), N2 = std::get<2>(go.second);
        const int sidx = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[sidx] += go.first;
        if (!use2(sidx)) return FENGINE_ECUDA;
        const cudaStream_t gs = b->pool[sidx];
        size_t rounds = 0;
        for (const auto *d : v) rounds = std::max(rounds, d->p1.size());
        for (size_t r = 0; r < rounds; r++) {
            std::vector<const fe::DeferredCall *> in;
            for (const auto *d : v)
                if (r < d->p1.size()) in.push_back(d);
            for (size_t a0 = 0; a0 < in.size(); a0 += fe::kMaxGroup) {
                const int nm = (int)std::min<size_t>(fe::kMaxGroup, in.size() - a0);
                fe::Phase1Group &g = *grouped;
                g.n = nm;
                int total = 0;
                for (int m = 0; m < nm; m++) {
                    const fe::DeferredCall &d = *in[a0 + m];
                    int gx = 0, gy = 0;
                    const int blocks = fe::phase1_blocks(d.N1, d.p1[r], d.n_streams, &gx, &gy);
                    g.p[m] = d.p1[r];
                    g.start[m] = total;
                    g.aux[m] = gy;
                    g.gx = gx;
                    total += blocks;
                }
                g.start[nm] = total;
                if (fe::launch_phase1_group(T, N1, g, gs) != cudaSuccess) return FENGINE_ECUDA;
                // the 1024-point stage is persistent: each member's CTAs in
                // proportion to its work within one wave
                fe::Phase2Group &g2 = *grouped2;
                g2.n = nm;
                long long items_all = 0;
                if (N2 == 1024)
                    for (int m = 0; m < nm; m++) items_all += fe::phase2w_items(in[a0 + m]->p2[r], in[a0 + m]->n_ant);
                total = 0;
                for (int m = 0; m < nm; m++) {
                    const fe::DeferredCall &d = *in[a0 + m];
                    int blocks = 0, gx = 1, gy = 1;
                    if (N2 == 1024) {
                        const long long items = fe::phase2w_items(d.p2[r], d.n_ant);
                        const long long c = items_all > 0 ? (long long)wave * items / items_all : 1;
                        blocks = (int)std::max(1LL, std::min(items, c));
                        gy = d.n_ant;   // aux: antennas
                    } else {
                        blocks = fe::phase2_blocks(N2, d.p2[r], d.n_ant, &gx, &gy);
                    }
                    g2.p[m] = d.p2[r];
                    g2.start[m] = total;
                    g2.aux[m] = gy;
                    g2.gx = gx;
                    total += blocks;
                }
                g2.start[nm] = total;
                if (fe::launch_phase2_group(N2, false, g2, gs) != cudaSuccess) return FENGINE_ECUDA;
            }
        }
    }
    // 5. join the pool's streams
    for (int s = 0; s < np; s++) {
        if (!used[s]) continue;
        if (cudaEventRecord(b->done[s], b->pool[s]) != cudaSuccess || cudaStreamWaitEvent(st, b->done[s], 0) != cudaSuccess)
            return FENGINE_ECUDA;
    }
    return result;
}

}  // extern "C"
