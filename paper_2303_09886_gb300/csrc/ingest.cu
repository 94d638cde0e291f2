// Host ingest (Sec. 3.1-3.2): digitiser heaps, in arrival order, into chunks
// on the device.
//
// The paper's receiver assembles heaps into chunks in host memory (each
// sample written by the NIC, read and written again by the assembly, read by
// the GPU copy) and pairs the two polarisations' chunks in Python. Here the
// host only appends each heap to a ring of pinned memory with a small
// descriptor (the one write a NIC's DMA would make); the ring goes to the
// device in arrival order on the ingest's own stream, as heaps come in, and
// a kernel scatters every heap to its place in the assembly chunk of its
// timestamp and sets its received flag. Both polarisations of every antenna
// share an assembly chunk, so pairing by timestamp is the chunk index, and a
// polarisation that lost heaps (or all of them) is just flagged (Sec. 3.7).
// Assembly chunks form a ring of reorder + 1 on the device: heaps of the
// next `reorder` chunks are accepted and placed while the oldest waits.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <algorithm>
#include <deque>
#include <new>
#include <utility>
#include <vector>

#include "../../include/fengine.h"

namespace {

struct Rec {
    int32_t slot, stream, heap, pad;   // assembly chunk, stream (2 antenna + pol), heap in the chunk
};

constexpr int kHeapVec = FENGINE_HEAP_BYTES / 16;   // 16-byte vectors per heap (320)

// One CTA per ring record [first, first + count) (positions modulo cap).
__global__ void __launch_bounds__(kHeapVec) k_heap_scatter(const uint8_t *__restrict__ ring,
                                                           const Rec *__restrict__ recs, int cap, long long first,
                                                           uint8_t *__restrict__ chunks, long long slot_bytes,
                                                           long long stream_bytes, uint8_t *__restrict__ valid,
                                                           int n_streams, int hpc) {
    const int pos = (int)((first + blockIdx.x) % cap);
    const Rec d = recs[pos];
    const uint4 *src = reinterpret_cast<const uint4 *>(ring + (size_t)pos * FENGINE_HEAP_BYTES);
    uint4 *dst = reinterpret_cast<uint4 *>(chunks + d.slot * slot_bytes + d.stream * stream_bytes +
                                           (long long)d.heap * FENGINE_HEAP_BYTES);
    dst[threadIdx.x] = src[threadIdx.x];
    if (threadIdx.x == 0) valid[((size_t)d.slot * n_streams + d.stream) * hpc + d.heap] = 1;
}

// Zero the samples of every heap of one assembly chunk that did not arrive
// (one CTA per (heap, stream)); they then read as zero in the channelizer.
__global__ void __launch_bounds__(kHeapVec) k_heap_zero_missing(uint8_t *__restrict__ chunk, long long stream_bytes,
                                                                const uint8_t *__restrict__ valid, int hpc) {
    const int h = blockIdx.x, s = blockIdx.y;
    if (valid[(size_t)s * hpc + h]) return;
    uint4 *dst = reinterpret_cast<uint4 *>(chunk + s * stream_bytes + (long long)h * FENGINE_HEAP_BYTES);
    dst[threadIdx.x] = make_uint4(0u, 0u, 0u, 0u);
}

}  // namespace

struct fengine_ingest_s {
    fengine_plan_t plan = nullptr;
    int n_streams = 0, hpc = 0, n_slots = 0, reorder = 0, cap = 0;
    long long L = 0, first = 0, stream_bytes = 0, slot_bytes = 0;
    // ring: positions are counted from 0 for ever, position p sits at p % cap
    uint8_t *h_ring = nullptr, *d_ring = nullptr;
    Rec *h_recs = nullptr, *d_recs = nullptr;
    long long head = 0;    // next position to write
    long long sent = 0;    // [.., sent) copied and scattered (enqueued)
    long long freed = 0;   // [.., freed) copies complete: reusable
    std::deque<std::pair<cudaEvent_t, long long>> inflight;   // copy-done event, end position
    std::vector<cudaEvent_t> spare;
    // assembly chunks on the device
    uint8_t *d_chunks = nullptr, *d_valid = nullptr;
    std::vector<std::vector<uint8_t>> got;   // per slot: received flags (host copy)
    std::vector<long long> count;            // per slot: heaps received
    long long next_emit = 0;
    bool blocked = false;                    // a push stopped at a heap past the reorder window
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_scat = nullptr, ev_done = nullptr;
    fengine_ingest_stats st{};
};

namespace {

cudaEvent_t take_event(fengine_ingest_s *g) {
    if (!g->spare.empty()) {
        cudaEvent_t e = g->spare.back();
        g->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

// ring positions whose device copy has completed become reusable
void reclaim(fengine_ingest_s *g, bool wait) {
    while (!g->inflight.empty()) {
        auto &f = g->inflight.front();
        if (wait) {
            if (cudaEventSynchronize(f.first) != cudaSuccess) return;
        } else if (cudaEventQuery(f.first) != cudaSuccess) {
            return;
        }
        g->freed = f.second;
        g->spare.push_back(f.first);
        g->inflight.pop_front();
    }
}

// copy ring positions [sent, head) to the device and scatter them
fengine_status send(fengine_ingest_s *g) {
    if (g->head == g->sent) return FENGINE_OK;
    const long long n = g->head - g->sent;
    const long long a = g->sent % g->cap;
    const long long n1 = n < g->cap - a ? n : g->cap - a;   // up to the end of the ring, then from 0
    const size_t hb = FENGINE_HEAP_BYTES;
    if (cudaMemcpyAsync(g->d_ring + a * hb, g->h_ring + a * hb, (size_t)n1 * hb, cudaMemcpyHostToDevice, g->cs) !=
            cudaSuccess ||
        cudaMemcpyAsync(g->d_recs + a, g->h_recs + a, (size_t)n1 * sizeof(Rec), cudaMemcpyHostToDevice, g->cs) !=
            cudaSuccess)
        return FENGINE_ECUDA;
    if (n1 < n && (cudaMemcpyAsync(g->d_ring, g->h_ring, (size_t)(n - n1) * hb, cudaMemcpyHostToDevice, g->cs) !=
                       cudaSuccess ||
                   cudaMemcpyAsync(g->d_recs, g->h_recs, (size_t)(n - n1) * sizeof(Rec), cudaMemcpyHostToDevice,
                                   g->cs) != cudaSuccess))
        return FENGINE_ECUDA;
    k_heap_scatter<<<(unsigned)n, kHeapVec, 0, g->cs>>>(g->d_ring, g->d_recs, g->cap, g->sent, g->d_chunks,
                                                         g->slot_bytes, g->stream_bytes, g->d_valid, g->n_streams,
                                                         g->hpc);
    if (cudaGetLastError() != cudaSuccess) return FENGINE_ECUDA;
    cudaEvent_t e = take_event(g);
    if (!e || cudaEventRecord(e, g->cs) != cudaSuccess) return FENGINE_ECUDA;
    g->inflight.emplace_back(e, g->head);
    g->st.bytes_to_device += n * (long long)(hb + sizeof(Rec));
    g->sent = g->head;
    return FENGINE_OK;
}

void release(fengine_ingest_s *g) {
    if (g->cs) cudaStreamSynchronize(g->cs);
    if (g->ev_done) cudaEventSynchronize(g->ev_done);   // the last emitted chunk has been read
    for (auto &f : g->inflight) cudaEventDestroy(f.first);
    for (cudaEvent_t e : g->spare) cudaEventDestroy(e);
    if (g->ev_scat) cudaEventDestroy(g->ev_scat);
    if (g->ev_done) cudaEventDestroy(g->ev_done);
    cudaFreeHost(g->h_ring);
    cudaFreeHost(g->h_recs);
    cudaFree(g->d_ring);
    cudaFree(g->d_recs);
    cudaFree(g->d_chunks);
    cudaFree(g->d_valid);
    if (g->cs) cudaStreamDestroy(g->cs);
    delete g;
}

}  // namespace

extern "C" fengine_status fengine_ingest_create(fengine_plan_t plan, int64_t first_sample, int32_t ring_heaps,
                                                int32_t reorder_chunks, fengine_ingest_t *out) {
    if (!plan || !out || ring_heaps < 1 || reorder_chunks < 0 || reorder_chunks > 3) return FENGINE_EINVAL;
    *out = nullptr;
    fengine_info info;
    if (fengine_get_info(plan, &info) != FENGINE_OK) return FENGINE_EINVAL;
    const long long N = 2LL * info.n_channels, L = info.spectra_per_chunk * N;
    if (L % FENGINE_HEAP_SAMPLES || first_sample % FENGINE_HEAP_SAMPLES || first_sample % N) return FENGINE_EINVAL;
    auto *g = new (std::nothrow) fengine_ingest_s;
    if (!g) return FENGINE_ENOMEM;
    g->plan = plan;
    g->n_streams = 2 * info.n_antennas;
    g->L = L;
    g->hpc = (int)(L / FENGINE_HEAP_SAMPLES);
    g->first = first_sample;
    g->reorder = reorder_chunks;
    g->n_slots = reorder_chunks + 1;
    g->cap = ring_heaps;
    g->stream_bytes = L / 4 * 5;
    g->slot_bytes = g->stream_bytes * g->n_streams;
    const size_t valid_bytes = (size_t)g->n_slots * g->n_streams * g->hpc;
    if (cudaHostAlloc((void **)&g->h_ring, (size_t)g->cap * FENGINE_HEAP_BYTES, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&g->h_recs, (size_t)g->cap * sizeof(Rec), cudaHostAllocDefault) != cudaSuccess ||
        cudaMalloc((void **)&g->d_ring, (size_t)g->cap * FENGINE_HEAP_BYTES) != cudaSuccess ||
        cudaMalloc((void **)&g->d_recs, (size_t)g->cap * sizeof(Rec)) != cudaSuccess ||
        cudaMalloc((void **)&g->d_chunks, (size_t)g->slot_bytes * g->n_slots) != cudaSuccess ||
        cudaMalloc((void **)&g->d_valid, valid_bytes) != cudaSuccess) {
        cudaGetLastError();
        release(g);
        return FENGINE_ENOMEM;
    }
    if (cudaStreamCreateWithFlags(&g->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_scat, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMemsetAsync(g->d_valid, 0, valid_bytes, g->cs) != cudaSuccess) {
        release(g);
        return FENGINE_ECUDA;
    }
    g->got.assign(g->n_slots, std::vector<uint8_t>((size_t)g->n_streams * g->hpc, 0));
    g->count.assign(g->n_slots, 0);
    *out = g;
    return FENGINE_OK;
}

extern "C" fengine_status fengine_ingest_destroy(fengine_ingest_t g) {
    if (!g) return FENGINE_EINVAL;
    release(g);
    return FENGINE_OK;
}

extern "C" fengine_status fengine_ingest_push(fengine_ingest_t g, const fengine_heap *heaps, int32_t n,
                                              int32_t *accepted) {
    if (!g || (n > 0 && !heaps) || n < 0 || !accepted) return FENGINE_EINVAL;
    *accepted = 0;
    for (int32_t i = 0; i < n; i++) {
        const fengine_heap &h = heaps[i];
        if (h.antenna < 0 || 2 * h.antenna >= g->n_streams || (h.pol != 0 && h.pol != 1) || !h.payload ||
            h.timestamp % FENGINE_HEAP_SAMPLES)
            return FENGINE_EINVAL;
        const long long rel = h.timestamp - g->first;
        if (rel < 0) {
            g->st.heaps_outside++;
            ++*accepted;
            continue;
        }
        const long long w = rel / g->L;
        if (w < g->next_emit) {
            g->st.heaps_late++;
            ++*accepted;
            continue;
        }
        if (w > g->next_emit + g->reorder) {
            g->blocked = true;
            return FENGINE_EBUSY;
        }
        const int slot = (int)(w % g->n_slots), stream = 2 * h.antenna + h.pol;
        const int hh = (int)((rel - w * g->L) / FENGINE_HEAP_SAMPLES);
        uint8_t &flag = g->got[slot][(size_t)stream * g->hpc + hh];
        if (flag) {
            g->st.heaps_duplicate++;
            ++*accepted;
            continue;
        }
        if (g->head - g->freed >= g->cap) {
            reclaim(g, false);
            if (g->head - g->freed >= g->cap) return FENGINE_EBUSY;   // ring full: poll first
        }
        const long long pos = g->head % g->cap;
        std::memcpy(g->h_ring + pos * FENGINE_HEAP_BYTES, h.payload, FENGINE_HEAP_BYTES);
        g->h_recs[pos] = Rec{slot, stream, hh, 0};
        g->head++;
        flag = 1;
        g->count[slot]++;
        g->st.heaps_accepted++;
        ++*accepted;
    }
    return FENGINE_OK;
}

extern "C" fengine_status fengine_ingest_poll(fengine_ingest_t g, void *cuda_stream, int32_t flush, int8_t *d_out,
                                              uint8_t *d_heap_flags, int32_t *emitted, int64_t *first_sample,
                                              int64_t *first_spectrum) {
    if (!g || !emitted) return FENGINE_EINVAL;
    *emitted = 0;
    fengine_status s = send(g);
    if (s != FENGINE_OK) return s;
    reclaim(g, false);
    const int slot = (int)(g->next_emit % g->n_slots);
    const bool complete = g->count[slot] == (long long)g->n_streams * g->hpc;
    const bool due = complete || flush || g->blocked;
    if (!due) return FENGINE_OK;
    if (!d_out) return FENGINE_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint8_t *chunk = g->d_chunks + (size_t)slot * g->slot_bytes;
    uint8_t *valid = g->d_valid + (size_t)slot * g->n_streams * g->hpc;
    // every scatter into the chunk precedes the processing
    if (cudaEventRecord(g->ev_scat, g->cs) != cudaSuccess || cudaStreamWaitEvent(st, g->ev_scat, 0) != cudaSuccess)
        return FENGINE_ECUDA;
    k_heap_zero_missing<<<dim3((unsigned)g->hpc, (unsigned)g->n_streams), kHeapVec, 0, st>>>(chunk, g->stream_bytes,
                                                                                          valid, g->hpc);
    if (cudaGetLastError() != cudaSuccess) return FENGINE_ECUDA;
    const long long t0 = g->first + g->next_emit * g->L;
    int64_t m0 = 0;
    s = fengine_process_chunk(g->plan, cuda_stream, chunk, t0, valid, d_out, d_heap_flags, nullptr, nullptr, &m0);
    if (s != FENGINE_OK) return s;
    // the slot is free for chunk next_emit + n_slots once the processing has read it
    if (cudaEventRecord(g->ev_done, st) != cudaSuccess || cudaStreamWaitEvent(g->cs, g->ev_done, 0) != cudaSuccess ||
        cudaMemsetAsync(valid, 0, (size_t)g->n_streams * g->hpc, g->cs) != cudaSuccess)
        return FENGINE_ECUDA;
    g->st.heaps_missing += (long long)g->n_streams * g->hpc - g->count[slot];
    g->st.chunks_emitted++;
    std::fill(g->got[slot].begin(), g->got[slot].end(), 0);
    g->count[slot] = 0;
    g->next_emit++;
    g->blocked = false;
    *emitted = 1;
    if (first_sample) *first_sample = t0;
    if (first_spectrum) *first_spectrum = m0;
    return FENGINE_OK;
}

extern "C" fengine_status fengine_ingest_get_stats(fengine_ingest_t g, fengine_ingest_stats *out) {
    if (!g || !out) return FENGINE_EINVAL;
    *out = g->st;
    return FENGINE_OK;
}
