// Small per-call kernels: the FP64 delay/phase table and the history-tail
// update, plus the phase-1 dispatch over tap counts.
#include "fe_device.cuh"
#include "fe_internal.cuh"

namespace fe {

template <int T>
cudaError_t launch_phase1_n1(int N1, const Phase1Params &p, int n_streams, cudaStream_t s);


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
    if (ci < 0 || ci > p.max_delay) {                    // unreachable after the host check
        ci = ci < 0 ? 0 : p.max_delay;
        atomicExch(p.err, 1);
    }
    p.ctab[e] = (int)ci;
    p.ftab[e] = make_float2((float)delta, (float)red);
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

}  // namespace fe
