// Small per-call kernels: the FP64 delay/phase table and the history-tail
// update, plus the phase-1 dispatch over tap counts.
#include "fe_device.cuh"
#include "fe_internal.cuh"

namespace fe {

template <int T>
cudaError_t launch_phase1_n1(int N1, const Phase1Params &p, int n_streams, cudaStream_t s);
template <int T>
cudaError_t launch_phase1_group_n1(int N1, const Phase1Group &g, cudaStream_t s);

cudaError_t launch_phase1_group(int T, int N1, const Phase1Group &g, cudaStream_t s) {
    switch (T) {
        case 1: return launch_phase1_group_n1<1>(N1, g, s);
        case 2: return launch_phase1_group_n1<2>(N1, g, s);
        case 4: return launch_phase1_group_n1<4>(N1, g, s);
        case 8: return launch_phase1_group_n1<8>(N1, g, s);
        case 16: return launch_phase1_group_n1<16>(N1, g, s);
        case 32: return launch_phase1_group_n1<32>(N1, g, s);
        default: return cudaErrorInvalidValue;
    }
}

// the grid launch_phase1 uses: (N2 / W, tiles of kP1Rows spectra, streams)
int phase1_blocks(int N1, const Phase1Params &p, int n_streams, int *gx, int *gy) {
    (void)N1;
    *gx = p.N2 / p.W;
    *gy = (p.q_count + kP1Rows - 1) / kP1Rows;
    return *gx * *gy * n_streams;
}


cudaError_t launch_phase1(int T, int N1, const Phase1Params &p, int n_streams, cudaStream_t s) {
    switch (T) {
        case 1: return launch_phase1_n1<1>(N1, p, n_streams, s);
        case 2: return launch_phase1_n1<2>(N1, p, n_streams, s);
        case 4: return launch_phase1_n1<4>(N1, p, n_streams, s);
        case 8: return launch_phase1_n1<8>(N1, p, n_streams, s);
        case 16: return launch_phase1_n1<16>(N1, p, n_streams, s);
        case 32: return launch_phase1_n1<32>(N1, p, n_streams, s);
        default: return cudaErrorInvalidValue;
    }
}

// Delay model per spectrum (Sec. 2.1 steps 2 and 4, Sec. 3.3): for the
// spectrum with timestamp t0 = N m, with the last segment whose t_apply <= t0
// (segment 0 before all of them),
//   d = d0 + rate (t0 - t_ref),  c = floor(d + 1/2),  delta = d - c,
//   phi = phi0 + phi_rate (t0 - t_ref).
// FP64 with explicit round-to-nearest operations (no contraction), so the
// host-side range check in the API computes the very same c. The phase is
// reduced to phi/pi in [-1, 1] before the single rounding to FP32.
__global__ void k_delay_table(const DelayTableParams p) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)p.n_streams * p.M) return;
    const int st = (int)(e / p.M), q = (int)(e % p.M);
    const long long t0 = (long long)p.N * (p.m0 + q);
    const DelaySeg *sg = p.seg + (long long)st * kMaxSeg;
    const int ns = p.nseg[st];
    int s = 0;
    for (int k = 0; k < ns; k++)
        if (sg[k].t_apply <= t0) s = k;
    const double dt = (double)(t0 - sg[s].t_ref);
    const double d = __dadd_rn(sg[s].d0, __dmul_rn(sg[s].rate, dt));
    const double c = floor(__dadd_rn(d, 0.5));
    const double delta = __dadd_rn(d, -c);
    const double phi = __dadd_rn(sg[s].phi0, __dmul_rn(sg[s].phi_rate, dt));
    const double u = phi * 0.31830988618379067154;       // phi / pi
    const double red = u - 2.0 * rint(0.5 * u);          // in [-1, 1]
    long long ci = (long long)c;
    if (ci < p.min_delay || ci > p.max_delay) {          // unreachable after the host check
        ci = ci < p.min_delay ? p.min_delay : p.max_delay;
        atomicExch(p.err, 1);
    }
    p.ctab[e] = (int)ci;
    p.ftab[e] = make_float2((float)delta, (float)red);
    if (p.cchg) {
        // the previous spectrum's coarse delay, recomputed the same way
        int chg = 0;
        if (q > 0) {
            const long long tp = t0 - p.N;
            int sp = 0;
            for (int k = 0; k < ns; k++)
                if (sg[k].t_apply <= tp) sp = k;
            const double dp = __dadd_rn(sg[sp].d0, __dmul_rn(sg[sp].rate, (double)(tp - sg[sp].t_ref)));
            long long cp = (long long)floor(__dadd_rn(dp, 0.5));
            cp = cp < p.min_delay ? p.min_delay : (cp > p.max_delay ? p.max_delay : cp);
            chg = cp != ci;
        }
        p.cchg[e] = (unsigned char)chg;
    }
    if (p.g_tapply) {
        const long long *ta = p.g_tapply + (long long)st * kMaxGainSeg;
        int g = 0;
        for (int k = 0; k < p.n_gsets[st]; k++)
            if (ta[k] <= t0) g = k;
        p.gsel[e] = (unsigned char)g;
    }
}

cudaError_t launch_delay_table(const DelayTableParams &p, cudaStream_t s) {
    const long long total = (long long)p.n_streams * p.M;
    const int threads = 256;
    const long long blocks = (total + threads - 1) / threads;
    k_delay_table<<<(unsigned)blocks, threads, 0, s>>>(p);
    return cudaGetLastError();
}

// New history = the last hist_bytes bytes of [old history | chunk] for every
// stream (the chunk-overlap region of Sec. 3.1, kept resident on the device
// instead of copying the next chunk's prefix).
__global__ void k_tail_update(const uint8_t *__restrict__ hist_in, const uint8_t *__restrict__ chunk,
                              uint8_t *__restrict__ hist_out, long long hist_bytes,
                              long long chunk_bytes, int n_streams) {
    const long long total = hist_bytes * n_streams;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long st = e / hist_bytes, b = e % hist_bytes;
        const long long src = b + chunk_bytes;
        hist_out[e] = src < hist_bytes ? hist_in[st * hist_bytes + src]
                                       : chunk[st * chunk_bytes + (src - hist_bytes)];
    }
}

cudaError_t launch_tail_update(const uint8_t *hist_in, const uint8_t *chunk, uint8_t *hist_out,
                               long long hist_bytes, long long chunk_bytes, int n_streams,
                               cudaStream_t s) {
    const long long total = hist_bytes * n_streams;
    long long blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_tail_update<<<(unsigned)blocks, 256, 0, s>>>(hist_in, chunk, hist_out, hist_bytes, chunk_bytes,
                                                   n_streams);
    return cudaGetLastError();
}

// Lost data (Sec. 3.7). Block x < n_ant * n_heaps_out: output heap h of
// antenna a; its threads check the spectra of the heap in both polarisations:
// spectrum m (coarse delay c) reads [N m - c, N m - c + N T), usable iff every
// heap that window touches was received (history heaps from hv_in, chunk
// heaps from valid). The heap is transmitted (flag 1) iff all are usable.
// The last block writes the received flags of the HV heaps before the end
// of this chunk, for the next call.
__global__ void k_lost_data(const LostDataParams p) {
    const int n_out = (p.M + p.S - 1) / p.S;
    const long long hist_first = p.heap0 - p.HV;   // heap of hv_in[0]
    auto received = [&](int stream, long long h) -> bool {
        if (h >= p.heap0) {
            const long long i = h - p.heap0;
            if (i >= p.chunk_heaps) return false;
            return p.valid ? p.valid[(long long)stream * p.chunk_heaps + i] != 0 : true;
        }
        const long long i = h - hist_first;
        return i >= 0 && p.hv_in[(long long)stream * p.HV + i] != 0;
    };
    if ((int)blockIdx.x < p.n_ant * n_out) {
        if (!p.heap_flags) return;
        const int a = blockIdx.x / n_out, h = blockIdx.x % n_out;
        const int q0 = h * p.S, cnt = min(p.S, p.M - q0);
        int ok = 1;
        for (int e = threadIdx.x; e < 2 * cnt; e += blockDim.x) {
            const int pol = e / cnt, q = q0 + e % cnt, stream = 2 * a + pol;
            const long long start = (long long)p.N * (p.m0 + q) - p.ctab[(long long)stream * p.M + q];
            const long long end = start + (long long)p.N * p.T - 1;
            const long long h0 = start >= 0 ? start / kHeapSamples : -((-start + kHeapSamples - 1) / kHeapSamples);
            const long long h1 = end >= 0 ? end / kHeapSamples : -((-end + kHeapSamples - 1) / kHeapSamples);
            for (long long hh = h0; hh <= h1 && ok; hh++)
                if (!received(stream, hh)) ok = 0;
        }
        ok = __syncthreads_and(ok);
        if (threadIdx.x == 0) p.heap_flags[(long long)a * n_out + h] = (unsigned char)ok;
        return;
    }
    // history heaps of the next call: heap (heap0 + chunk_heaps) - HV + i
    for (int e = threadIdx.x; e < 2 * p.n_ant * p.HV; e += blockDim.x) {
        const int stream = e / p.HV, i = e % p.HV;
        const long long hh = p.heap0 + p.chunk_heaps - p.HV + i;
        p.hv_out[(long long)stream * p.HV + i] = received(stream, hh) ? 1 : 0;
    }
}

cudaError_t launch_lost_data(const LostDataParams &p, cudaStream_t s) {
    const int n_out = (p.M + p.S - 1) / p.S;
    k_lost_data<<<p.n_ant * n_out + 1, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace fe
