// Phase 2, reduced-precision form (N2 = 1024): the second stage of the
// four-step DFT as two 32-point DFT contractions on tensor cores
// (mma.sync m16n8k16, FP16 or BF16 operands, FP32 accumulation), then the
// fine-delay rotation, gain, requantisation and corner turn of the FP32
// form (Sec. 2.1 steps 4-6, Sec. 2.2, Sec. 3.6).
//
// With t2 = 32 a + b and k2 = c + 32 d (a, b, c, d in [0, 32)):
//   Y[c][b]     = sum_a exp(-2 pi i c a / 32) B[32 a + b]        (contraction 1)
//   Y'[c][b]    = exp(-2 pi i c b / 1024) Y[c][b]                (twiddle)
//   F[c + 32 d] = sum_b Y'[c][b] exp(-2 pi i d b / 32)           (contraction 2)
// Each contraction is a real 64 x 64 product over (index, re/im) pairs.
// Contraction 1 has the DFT matrix as operand A (rows: c, re/im) and the
// data as operand B (columns: b); contraction 2 has the data as operand A
// (rows: c) and the DFT matrix as operand B (columns: d, re/im). Inside a
// 16-wide K tile, positions 2q + e and 2q + 8 + e (q < 4, e = re/im) hold
// index 8 kt + 2q and 8 kt + 2q + 1. With that order the accumulator of
// contraction 1 -- lane (g, q) holds Y[8 mt + g][8 nt + 2q + {0, 1}] -- is,
// after the twiddle and rounding, exactly lane (g, q)'s operand A of
// contraction 2: the data never leaves the registers between the two.
//
// One CTA owns one class k1 and 8 consecutive spectra of both polarisations
// of one antenna; warp w computes spectrum w, one polarisation after the
// other. The DFT matrices (as per-lane fragments) and the twiddles come from
// plan tables; scale factors keep every FP16 operand below 2^15: the plan
// scales the first-stage twiddle by s1 (from the weights' bound), the
// twiddle table carries 2^-5 (contraction 1 grows values by at most 32),
// and the rotation tables carry the inverse of both.
//
// Split operands: an operand x is carried as hi = round(x) and lo =
// round(x - hi) in the operand type, and a product as hi.hi + hi.lo + lo.hi,
// which leaves an error of the order of the type's precision squared. A
// strong tone makes one class sequence far larger than its neighbours in
// the spectrum, and a single rounding of the DFT matrices or of the data
// between the contractions puts an error of a few 1e-4 of the tone's
// amplitude into every channel of the class: several 8-bit LSB next to a
// tone that saturates. So both forms split the DFT matrices and the data
// between the contractions. The FP16 form's input B is already an FP16
// value (the intermediate is stored in FP16) and needs no split:
// contraction 1 takes 2 products there, contraction 2 takes 3. The BF16
// form splits its FP32 input as well (3 and 3).
#include <cmath>
#include <cstring>
#include <type_traits>

#include "fe_device.cuh"
#include "fe_internal.cuh"
#include "fe_mma.cuh"

namespace fe {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcR = 8;          // spectra per CTA, one warp each
constexpr int kTcN2 = 1024;
constexpr int kGainLd = kTcN2 + kTcN2 / 8;   // padded gain row (conflict-free 8-byte loads)
constexpr int kPQ = 65;                      // per sequence: P[32], Q[32], qu
constexpr int kStgLd = kTcN2 + kTcN2 / 4 + 4; // staging row stride in words (= 4 mod 32)

// Padded slots. A lane (g, q) of the epilogue handles k2 = g + 32 q + const
// (const < 32 apart from multiples of 128), so (k2 >> 5) = q + const / 32:
//   gain slot    k2 + 4 (k2 >> 5)  -> 8-byte loads without bank conflicts,
//   staging word k2 + 8 (k2 >> 5)  -> 2-byte stores without bank conflicts,
// and the row stride kStgLd = 4 (mod 32) keeps the corner-turn reads (four
// spectra of one slot per thread) conflict-free as well.
__device__ __forceinline__ int gain_slot(int k2) { return k2 + 4 * (k2 >> 5); }
__device__ __forceinline__ int stage_slot(int k2) { return k2 + 8 * (k2 >> 5); }

}  // namespace

// shared memory: tables (hi and lo) + P/Q + gains + staging + row info
size_t phase2_tc_smem_bytes(int) {
    const int nl = 2;
    const size_t pq = (sizeof(float2) * 2 * kTcR * kPQ + 15) / 16 * 16;
    return sizeof(uint4) * 512 * (1 + 2 * nl) + pq + sizeof(float2) * 2 * kGainLd +
           sizeof(unsigned) * kStgLd * kTcR + (sizeof(long long) + sizeof(int)) * kTcR;
}

template <int PREC>
__global__ void __launch_bounds__(kTcThreads, 2) k_phase2_tc(const Phase2Params p) {
    extern __shared__ uint4 smu[];
    // plan table order: a1 [4 mt][4 kt][32], b2 [4 kt2][4 ntp][32], tw [4 mt][4 nt][32], a1 lo, b2 lo
    const uint4 *a1s = smu, *b2s = smu + 512;
    const float4 *tws = reinterpret_cast<const float4 *>(smu + 1024);
    const uint4 *a1l = smu + 1536, *b2l = smu + 2048;
    float2 *pq = reinterpret_cast<float2 *>(smu + 2560);                  // [2 kTcR][kPQ]
    float2 *gsm = pq + (2 * kTcR * kPQ + 1) / 2 * 2;                     // [2][kGainLd]
    unsigned *stg = reinterpret_cast<unsigned *>(gsm + 2 * kGainLd);     // [kTcR][kStgLd]
    long long *rowoff = reinterpret_cast<long long *>(stg + kStgLd * kTcR);
    int *rowstride = reinterpret_cast<int *>(rowoff + kTcR);

    const int k1 = blockIdx.x, ant = blockIdx.z;
    const int q0 = p.q_begin + blockIdx.y * kTcR;
    const int M = p.M, Rv = min(kTcR, p.q_begin + p.q_count - q0);
    const int N1 = p.N1, H1 = N1 / 2, N = p.N, n = N / 2, S_ = p.S;
    const bool upper = (k1 != 0 && k1 != H1);
    const int nslot = upper ? kTcN2 : kTcN2 / 2;

    for (int i = threadIdx.x; i < 2560; i += kTcThreads) smu[i] = __ldg(p.tc + i);
    // rotation factors of each (pol, spectrum) sequence, angles over pi:
    //   P[c] = u exp(i pi (phi/pi - 2 delta (k1 + N1 c) / N)),
    //   Q[d] = exp(-i pi 2 delta 32 N1 d / N),  qu = exp(i pi (2 phi/pi - 2 delta)),
    // so that channel k1 + N1 k2 (k2 = c + 32 d) is P[c] Q[d] F[k2] and the
    // upper-half channel N - (k1 + N1 k2) is qu conj(P[c] Q[d] F[k2]).
    const float inv = 2.0f / (float)N, u = p.tc_unscale;
    for (int e = threadIdx.x; e < 2 * kTcR * kPQ; e += kTcThreads) {
        const int sq = e / kPQ, j = e - sq * kPQ;
        const int pol = sq / kTcR, r = sq % kTcR;
        if (r >= Rv) continue;
        const float2 f = p.ftab[(long long)(ant * 2 + pol) * M + q0 + r];   // (delta, phi / pi)
        const int c = j & 31;
        float ang, sc = 1.0f;
        if (j < 32) {
            ang = f.y - f.x * (float)(k1 + N1 * c) * inv;
            sc = u;
        } else if (j < 64) {
            ang = -f.x * (float)(32 * N1 * c) * inv;
        } else {
            ang = 2.0f * f.y - 2.0f * f.x;
        }
        float sn, cs;
        sincospif(ang, &sn, &cs);
        pq[e] = make_float2(sc * cs, sc * sn);
    }
    // gains of this CTA's slots (slot k2 is channel k1 + N1 k2 in the lower
    // half, N - (k1 + N1 k2) in the upper)
    for (int e = threadIdx.x; e < 2 * kTcN2; e += kTcThreads) {
        const int pol = e / kTcN2, k2 = e % kTcN2;
        const int kc = k1 + N1 * k2;
        const int k = k2 >= kTcN2 / 2 ? N - kc : kc;
        gsm[pol * kGainLd + gain_slot(k2)] =
            (k >= 0 && k < n) ? __ldg(p.gains + (long long)(ant * 2 + pol) * n + k) : make_float2(0.f, 0.f);
    }
    if ((int)threadIdx.x < Rv) {
        const int q = q0 + threadIdx.x;
        const int h = q / S_, s = q - h * S_;
        const int Sh = min(S_, M - h * S_);
        rowoff[threadIdx.x] = (long long)h * S_ * n * 4 + s * 4;
        rowstride[threadIdx.x] = Sh * 4;
    }
    __syncthreads();

    const int r = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    unsigned short *stg16 = reinterpret_cast<unsigned short *>(stg);
    if (r < Rv) {
        for (int pol = 0; pol < 2; pol++) {
            const int stream = ant * 2 + pol;
            const long long base = ((long long)(stream * p.a_spectra + (q0 - p.q_begin) + r) * (H1 + 1) + k1) * kTcN2;
            const float2 *pqs = pq + (pol * kTcR + r) * kPQ;
            const float2 qu = pqs[64];
            float2 *pre = p.prequant ? p.prequant + ((long long)stream * M + q0 + r) * n : nullptr;
            // lane parts of the gain slot and staging slot of k2 = g + 32 tq + 16 mp + 8 h + 128 nt2
            const float2 *gp = gsm + pol * kGainLd + g + 36 * tq;
            unsigned short *sp = stg16 + 2 * (r * kStgLd + g + 40 * tq) + pol;
            // The lane's operands B of contraction 1: K tile kt takes B[32 a + b]
            // at a = 8 kt + 2 tq + h, b = 8 nt + g. FP16 form: the intermediate
            // holds the (re, im) FP16 pairs the products take; all four K tiles
            // are loaded per row half (128 registers a thread leave no room to
            // keep them across both). BF16 form: FP32 pairs, one K tile at a
            // time (below).
            using In = std::conditional_t<PREC == 1, unsigned, float2>;
            const In *src = reinterpret_cast<const In *>(p.A) + base;
            [[maybe_unused]] unsigned v[4][4][2];
            // Rows c = 16 mp + (0 .. 15) of Y' need only m tiles 2 mp and
            // 2 mp + 1 of contraction 1, and give rows c of F: both
            // contractions and the epilogue run per mp, so that only half of
            // the first accumulator is live at a time.
#pragma unroll
            for (int mp = 0; mp < 2; mp++) {
                if constexpr (PREC == 1) {
#pragma unroll
                    for (int kt = 0; kt < 4; kt++)
#pragma unroll
                        for (int nt = 0; nt < 4; nt++)
#pragma unroll
                            for (int h = 0; h < 2; h++) v[kt][nt][h] = __ldg(src + 32 * (8 * kt + 2 * tq + h) + 8 * nt + g);
                }
                float d1[2][4][4];
#pragma unroll
                for (int i = 0; i < 2; i++)
#pragma unroll
                    for (int nt = 0; nt < 4; nt++)
#pragma unroll
                        for (int x = 0; x < 4; x++) d1[i][nt][x] = 0.0f;
                if constexpr (PREC == 1) {
#pragma unroll
                    for (int kt = 0; kt < 4; kt++) {
#pragma unroll
                        for (int i = 0; i < 2; i++) {
                            const int mt = 2 * mp + i;
                            const uint4 A = a1s[(mt * 4 + kt) * 32 + lane], Al = a1l[(mt * 4 + kt) * 32 + lane];
#pragma unroll
                            for (int nt = 0; nt < 4; nt++) {
                                mma16816<PREC>(d1[i][nt], A, v[kt][nt][0], v[kt][nt][1]);
                                mma16816<PREC>(d1[i][nt], Al, v[kt][nt][0], v[kt][nt][1]);
                            }
                        }
                    }
                } else {
                    // FP32 pairs one K tile at a time (the next tile's loads in
                    // flight), split into hi and lo here: 3 products
                    float2 vk[2][4][2];
                    auto load_kt = [&](int kt, float2 (&dst)[4][2]) {
#pragma unroll
                        for (int nt = 0; nt < 4; nt++)
#pragma unroll
                            for (int h = 0; h < 2; h++) dst[nt][h] = __ldg(src + 32 * (8 * kt + 2 * tq + h) + 8 * nt + g);
                    };
                    load_kt(0, vk[0]);
#pragma unroll
                    for (int kt = 0; kt < 4; kt++) {
                        if (kt < 3) load_kt(kt + 1, vk[(kt + 1) & 1]);
                        unsigned bh[4][2], bl[4][2];
#pragma unroll
                        for (int nt = 0; nt < 4; nt++)
#pragma unroll
                            for (int h = 0; h < 2; h++) {
                                const float2 x = vk[kt & 1][nt][h];
                                bh[nt][h] = pack2<PREC>(x.x, x.y);
                                bl[nt][h] = pack2<PREC>(x.x - prec_round<PREC>(x.x), x.y - prec_round<PREC>(x.y));
                            }
#pragma unroll
                        for (int i = 0; i < 2; i++) {
                            const int mt = 2 * mp + i;
                            const uint4 A = a1s[(mt * 4 + kt) * 32 + lane], Al = a1l[(mt * 4 + kt) * 32 + lane];
#pragma unroll
                            for (int nt = 0; nt < 4; nt++) {
                                mma16816<PREC>(d1[i][nt], A, bh[nt][0], bh[nt][1]);
                                mma16816<PREC>(d1[i][nt], Al, bh[nt][0], bh[nt][1]);
                                mma16816<PREC>(d1[i][nt], A, bl[nt][0], bl[nt][1]);
                            }
                        }
                    }
                }
                // twiddle; lane (g, tq) then holds operand A of contraction 2
                // for K tile kt2 (b = 8 kt2 + 2 tq, + 1) and rows c = 16 mp + g, + 8:
                // a0 = Y'[c][b], a1 = Y'[c + 8][b], a2 = Y'[c][b + 1], a3 = Y'[c + 8][b + 1]
                unsigned ah[4][4], al[4][4];
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    const int mt = 2 * mp + i;
#pragma unroll
                    for (int nt = 0; nt < 4; nt++) {
                        const float4 t = tws[(mt * 4 + nt) * 32 + lane];
                        const float2 y0 = cmul(make_float2(d1[i][nt][0], d1[i][nt][2]), make_float2(t.x, t.y));
                        const float2 y1 = cmul(make_float2(d1[i][nt][1], d1[i][nt][3]), make_float2(t.z, t.w));
                        ah[nt][i] = pack2<PREC>(y0.x, y0.y);
                        ah[nt][2 + i] = pack2<PREC>(y1.x, y1.y);
                        al[nt][i] = pack2<PREC>(y0.x - prec_round<PREC>(y0.x), y0.y - prec_round<PREC>(y0.y));
                        al[nt][2 + i] = pack2<PREC>(y1.x - prec_round<PREC>(y1.x), y1.y - prec_round<PREC>(y1.y));
                    }
                }
                // contraction 2 and the epilogue per half of the output
                // columns (d < 16: lower-half channels, d >= 16: upper)
#pragma unroll
                for (int half = 0; half < 2; half++) {
                    if (half == 1 && !upper) break;
                    float d2[4][4];
#pragma unroll
                    for (int j = 0; j < 4; j++)
#pragma unroll
                        for (int x = 0; x < 4; x++) d2[j][x] = 0.0f;
#pragma unroll
                    for (int kt2 = 0; kt2 < 4; kt2++) {
#pragma unroll
                        for (int jp = 0; jp < 2; jp++) {
                            const int ntp = 2 * half + jp;
                            const uint4 B = b2s[(kt2 * 4 + ntp) * 32 + lane];
                            const uint4 Bl = b2l[(kt2 * 4 + ntp) * 32 + lane];
                            mma16816<PREC>(d2[2 * jp], ah[kt2], B.x, B.y);
                            mma16816<PREC>(d2[2 * jp + 1], ah[kt2], B.z, B.w);
                            mma16816<PREC>(d2[2 * jp], ah[kt2], Bl.x, Bl.y);
                            mma16816<PREC>(d2[2 * jp + 1], ah[kt2], Bl.z, Bl.w);
                            mma16816<PREC>(d2[2 * jp], al[kt2], B.x, B.y);
                            mma16816<PREC>(d2[2 * jp + 1], al[kt2], B.z, B.w);
                        }
                    }
                    // rotation, gain, requantisation into the staging cells
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int cl = 16 * mp + 8 * h;          // c = cl + g
                        float2 Pc = pqs[cl + g];
                        if (half == 1) Pc = cmul(qu, cconj(Pc));
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const int nt2 = 4 * half + j;
                            float2 rot = pqs[32 + 4 * nt2 + tq];
                            rot = half == 0 ? cmul(Pc, rot) : cmul(Pc, cconj(rot));
                            float2 F = make_float2(d2[j][2 * h], d2[j][2 * h + 1]);
                            if (half == 1) F = cconj(F);
                            const float2 y = cmul(gp[cl + 144 * nt2], cmul(rot, F));
                            if (pre) {
                                const int k2 = cl + g + 32 * (4 * nt2 + tq);
                                pre[half == 0 ? k1 + N1 * k2 : N - (k1 + N1 * k2)] = y;
                            }
                            sp[2 * (cl + 160 * nt2)] =
                                (unsigned short)__byte_perm((unsigned)quant8(y.x), (unsigned)quant8(y.y), 0x0040u);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();

    // corner turn: cell (slot k2, spectrum r) -> heap row of channel k. When
    // each group of four spectra shares a heap and its cells are 16-byte
    // aligned (spectra per heap and the heap's size multiples of 4), a thread
    // writes four spectra of a slot with one 16-byte store.
    int8_t *out = p.out + (long long)ant * M * n * 4;
    const bool vec = Rv == kTcR && S_ % 4 == 0 && rowstride[0] % 16 == 0 && rowstride[4] % 16 == 0;
    if (vec) {
        for (int e = threadIdx.x; e < nslot * 2; e += kTcThreads) {
            const int k2 = e >> 1, r4 = 4 * (e & 1);
            const int kc = k1 + N1 * k2;
            const int k = k2 >= kTcN2 / 2 ? N - kc : kc;
            const unsigned *cell = stg + r4 * kStgLd + stage_slot(k2);
            const uint4 v = make_uint4(cell[0], cell[kStgLd], cell[2 * kStgLd], cell[3 * kStgLd]);
            *reinterpret_cast<uint4 *>(out + rowoff[r4] + (long long)k * rowstride[r4]) = v;
        }
    } else {
        for (int e = threadIdx.x; e < nslot * kTcR; e += kTcThreads) {
            const int k2 = e / kTcR, rr = e % kTcR;
            if (rr >= Rv) continue;
            const int kc = k1 + N1 * k2;
            const int k = k2 >= kTcN2 / 2 ? N - kc : kc;
            *reinterpret_cast<unsigned *>(out + rowoff[rr] + (long long)k * rowstride[rr]) =
                stg[rr * kStgLd + stage_slot(k2)];
        }
    }
}

// ---- host: the plan tables

namespace {

// Contraction 1's operand A: row m = 16 mt + 8 o + i is output c = 8 mt + i
// (o = 0 real, 1 imaginary part); K position 16 kt + p is input
// a = 8 kt + 2 ((p & 7) >> 1) + (p >> 3), part p & 1. The block of the real
// form of exp(-2 pi i c a / 32) = C - i S is [[C, S], [-S, C]].
double dft_block(int idx_prod, int out_im, int in_im) {
    const double th = 2.0 * M_PI * (double)(idx_prod % 32) / 32.0;
    const double C = std::cos(th), S = std::sin(th);
    if (!out_im) return in_im ? S : C;
    return in_im ? C : -S;
}

int k_index(int k) { return 8 * (k / 16) + 2 * ((k % 16 & 7) >> 1) + ((k % 16) >> 3); }

double a1_value(int m, int k) {
    const int c = 8 * (m / 16) + (m % 16 & 7);
    return dft_block(c * k_index(k), (m % 16) >> 3, k & 1);
}

// Contraction 2's operand B: K position as above (input b), column
// n = 8 nt + l is output d = 4 nt + (l >> 1), part l & 1.
double b2_value(int k, int n) {
    const int d = 4 * (n / 8) + ((n % 8) >> 1);
    return dft_block(d * k_index(k), n & 1, k & 1);
}

// Two matrix entries as one 32-bit operand register (first entry in the low
// half); part 0 is the rounded value, part 1 the rounded remainder.
unsigned pack_pair(double v0, double v1, int precision, int part) {
    unsigned short h[2];
    const double v[2] = {v0, v1};
    for (int i = 0; i < 2; i++) {
        if (precision == 1) {
            __half x = __float2half_rn((float)v[i]);
            if (part) x = __float2half_rn((float)(v[i] - (double)__half2float(x)));
            std::memcpy(&h[i], &x, 2);
        } else {
            __nv_bfloat16 x = __float2bfloat16_rn((float)v[i]);
            if (part) x = __float2bfloat16_rn((float)(v[i] - (double)__bfloat162float(x)));
            std::memcpy(&h[i], &x, 2);
        }
    }
    return (unsigned)h[0] | ((unsigned)h[1] << 16);
}

}  // namespace

void build_phase2_tc_tables(int precision, uint4 *out) {
    std::memset(out, 0, sizeof(uint4) * kPhase2TcTableLen);
    for (int part = 0; part < 2; part++) {
        uint4 *a1 = out + (part ? 1536 : 0), *b2 = out + (part ? 2048 : 512);
        for (int lane = 0; lane < 32; lane++) {
            const int g = lane >> 2, q = lane & 3;
            for (int mt = 0; mt < 4; mt++)
                for (int kt = 0; kt < 4; kt++) {
                    const int r0 = 16 * mt + g, c0 = 16 * kt + 2 * q;
                    uint4 f;
                    f.x = pack_pair(a1_value(r0, c0), a1_value(r0, c0 + 1), precision, part);
                    f.y = pack_pair(a1_value(r0 + 8, c0), a1_value(r0 + 8, c0 + 1), precision, part);
                    f.z = pack_pair(a1_value(r0, c0 + 8), a1_value(r0, c0 + 9), precision, part);
                    f.w = pack_pair(a1_value(r0 + 8, c0 + 8), a1_value(r0 + 8, c0 + 9), precision, part);
                    a1[(mt * 4 + kt) * 32 + lane] = f;
                }
            for (int kt = 0; kt < 4; kt++)
                for (int ntp = 0; ntp < 4; ntp++) {
                    const int k0 = 16 * kt + 2 * q;
                    unsigned v[4];
                    for (int j = 0; j < 2; j++) {
                        const int col = 8 * (2 * ntp + j) + g;
                        v[2 * j] = pack_pair(b2_value(k0, col), b2_value(k0 + 1, col), precision, part);
                        v[2 * j + 1] = pack_pair(b2_value(k0 + 8, col), b2_value(k0 + 9, col), precision, part);
                    }
                    b2[(kt * 4 + ntp) * 32 + lane] = make_uint4(v[0], v[1], v[2], v[3]);
                }
        }
    }
    // twiddle exp(-2 pi i c b / 1024) 2^-5 at c = 8 mt + g, b = 8 nt + 2 q + e
    for (int lane = 0; lane < 32; lane++) {
        const int g = lane >> 2, q = lane & 3;
        for (int mt = 0; mt < 4; mt++)
            for (int nt = 0; nt < 4; nt++) {
                float t[4];
                for (int e = 0; e < 2; e++) {
                    const int c = 8 * mt + g, b = 8 * nt + 2 * q + e;
                    const double th = 2.0 * M_PI * (double)((c * b) % kTcN2) / (double)kTcN2;
                    t[2 * e] = (float)(std::cos(th) / 32.0);
                    t[2 * e + 1] = (float)(-std::sin(th) / 32.0);
                }
                std::memcpy(&out[1024 + (mt * 4 + nt) * 32 + lane], t, sizeof(t));
            }
    }
}

cudaError_t launch_phase2_tc(const Phase2Params &p, int n_ant, cudaStream_t s) {
    if (p.N / p.N1 != kTcN2 || !p.tc || (p.precision != 1 && p.precision != 2)) return cudaErrorInvalidValue;
    const size_t smem = phase2_tc_smem_bytes(p.precision);
    dim3 grid(p.N1 / 2 + 1, (p.q_count + kTcR - 1) / kTcR, n_ant);
    cudaError_t e;
    if (p.precision == 1) {
        if ((e = cudaFuncSetAttribute(k_phase2_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        k_phase2_tc<1><<<grid, kTcThreads, smem, s>>>(p);
    } else {
        if ((e = cudaFuncSetAttribute(k_phase2_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        k_phase2_tc<2><<<grid, kTcThreads, smem, s>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace fe
