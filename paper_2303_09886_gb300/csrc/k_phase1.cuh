// Phase 1 of the fused F-engine: 10-bit unpack, coarse delay, PFB FIR (Eq. 1)
// and the first stage of the four-step real DFT.
//
// Four-step split of the N-point DFT of one spectrum's filtered samples g:
//   t = N2 t1 + t2, k = k1 + N1 k2,
//   X[k1 + N1 k2] = sum_t2 exp(-2 pi i k2 t2 / N2) * B[k1][t2],
//   B[k1][t2]     = exp(-2 pi i k1 t2 / N) * sum_t1 g[N2 t1 + t2] exp(-2 pi i k1 t1 / N1).
// g is real, so only k1 in [0, N1/2] is kept (the rest is the conjugate).
//
// One CTA owns a tile of kP1Rows consecutive spectra x C = N1 * W columns
// {N2 t1 + t2 : t1 < N1, t2 in [t2_0, t2_0 + W)} of one (antenna, pol)
// stream. It
//   1. unpacks the (kP1Rows + T - 1) rows of delayed samples the tile needs
//      into shared memory as FP32 (exact for 10-bit integers), one run of
//      constant coarse delay at a time (Sec. 3.3: each PFB window uses one
//      consistent delay);
//   2. runs the T-tap FIR down each column with the weights and a sliding
//      window of T samples in registers (one shared-memory load and T FMAs
//      per output), writing g in place;
//   3. for each (spectrum, t2) does the real N1-point DFT over t1 in
//      registers (an N1/2-point complex FFT of even/odd pairs plus the
//      split), multiplies by the twiddle and stores B to the intermediate.
#pragma once
#include "fe_device.cuh"
#include "fe_internal.cuh"

namespace fe {

template <int T, int N1>
__global__ void __launch_bounds__(512) k_phase1(const Phase1Params p) {
    constexpr int R = kP1Rows;
    constexpr int H1 = N1 / 2;
    extern __shared__ float xs[];              // [(R + T - 1)][C]
    __shared__ int c_sm[R];
    __shared__ float2 tw_sm[33];               // exp(-2 pi i q / 64)

    const int C = p.C, W = p.W, N = p.N, N2 = p.N2;
    const int stream = blockIdx.z;
    const int t2_0 = blockIdx.x * W;
    const int q0 = blockIdx.y * R;
    const int Rv = min(R, p.M - q0);
    const uint8_t *chunk = p.chunk + (long long)stream * p.chunk_bytes;
    const uint8_t *hist = p.hist + (long long)stream * p.hist_bytes;
    const long long base = p.t_in - p.H;       // absolute index of history sample 0

    for (int i = threadIdx.x; i < Rv; i += blockDim.x) c_sm[i] = p.ctab[(long long)stream * p.M + q0 + i];
    for (int i = threadIdx.x; i < 33; i += blockDim.x) {
        float s, c;
        sincospif(-(float)i / 32.0f, &s, &c);
        tw_sm[i] = make_float2(c, s);
    }
    __syncthreads();

    int ra = 0;
    while (ra < Rv) {
        const int cd = c_sm[ra];
        int rb = ra + 1;
        while (rb < Rv && c_sm[rb] == cd) rb++;
        // 1. delayed samples for rows [ra, rb + T - 1)
        const int rows = rb + T - 1 - ra;
        for (int e = threadIdx.x; e < rows * C; e += blockDim.x) {
            const int row = ra + e / C, col = e % C;
            const int t = N2 * (col / W) + t2_0 + (col % W);
            const long long i = (long long)N * (p.m0 + q0 + row) - cd + t;
            const long long rel = i - base;
            const int v = rel < p.H ? fetch10(hist, rel) : fetch10(chunk, rel - p.H);
            xs[row * C + col] = (float)v;
            if (p.window_tap && row < rb)
                p.window_tap[((long long)stream * p.M + q0 + row) * N + t] = v;
        }
        __syncthreads();
        // 2. FIR down each column, g written over the row it starts at
        for (int col = threadIdx.x; col < C; col += blockDim.x) {
            const int t = N2 * (col / W) + t2_0 + (col % W);
            float wr[T], win[T];
#pragma unroll
            for (int j = 0; j < T; j++) wr[j] = __ldg(p.w + t + (long long)N * j);
#pragma unroll
            for (int row = 0; row < R + T - 1; row++) {
                if (row >= ra && row < rb + T - 1) win[row % T] = xs[row * C + col];
                const int r = row - (T - 1);
                if (r >= ra && r < rb) {
                    float acc = 0.0f;
#pragma unroll
                    for (int j = 0; j < T; j++) acc = fmaf(wr[j], win[(r + j) % T], acc);
                    xs[r * C + col] = acc;
                }
            }
        }
        __syncthreads();
        ra = rb;
    }

    // 3. real N1-point DFT over t1, twiddle, store B[k1][t2]
    for (int pi = threadIdx.x; pi < Rv * W; pi += blockDim.x) {
        const int r = pi / W, w = pi % W;
        const float *g = xs + r * C + w;
        float2 z[H1];
#pragma unroll
        for (int q = 0; q < H1; q++) z[q] = make_float2(g[(2 * q) * W], g[(2 * q + 1) * W]);
        fft_reg<H1>(z, tw_sm);
        const int t2 = t2_0 + w;
        float2 *out = p.A + ((long long)stream * p.M + q0 + r) * (H1 + 1) * N2 + t2;
#pragma unroll
        for (int k = 0; k <= H1; k++) {
            const float2 zk = z[k % H1], zm = z[(H1 - k) % H1];
            // even part E = (Z[k] + conj Z[H1-k]) / 2, odd part O = (Z[k] - conj Z[H1-k]) / 2i
            const float2 E = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            const float2 O = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
            const float2 a = cadd(E, cmul(tw_sm[k * (64 / N1)], O));
            out[(long long)k * N2] = cmul(a, __ldg(p.tw1 + (long long)k * N2 + t2));
        }
    }
}

template <int T, int N1>
cudaError_t launch_phase1_t(const Phase1Params &p, int n_streams, cudaStream_t s) {
    const int threads = p.C < 512 ? p.C : 512;
    const size_t smem = phase1_smem_bytes(T, p.C);
    cudaError_t e = cudaFuncSetAttribute(k_phase1<T, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(p.N2 / p.W, (p.M + kP1Rows - 1) / kP1Rows, n_streams);
    k_phase1<T, N1><<<grid, threads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int T>
cudaError_t launch_phase1_n1(int N1, const Phase1Params &p, int n_streams, cudaStream_t s) {
    switch (N1) {
        case 8: return launch_phase1_t<T, 8>(p, n_streams, s);
        case 16: return launch_phase1_t<T, 16>(p, n_streams, s);
        case 32: return launch_phase1_t<T, 32>(p, n_streams, s);
        case 64: return launch_phase1_t<T, 64>(p, n_streams, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fe
