// pfb_general.cu -- the PFB of Sec. III.A for channel counts that are not a
// power of two, or too large for one CTA (Fig. 3 channelizes with N = 10^5;
// the section reports up to 10^7 bins): any N = 2^a 3^b 5^c 7^d with
// 2 <= N <= 2^24, T <= 16 taps per channel, any hop 1 <= H <= N between frames.
//
// Frame k of the virtual stream [carry | buffer] uses the T*N samples from
// k*H on (H = hop, N when critically sampled):
//   v_k[p] = sum_{t<T} h[t*N + p] * x[k*H + t*N + p],
//   y_k[c] = sum_p v_k[p] exp(-2*pi*i*c*(A_k + p)/N),
// A_k the absolute index of the window's first sample (a multiple of N when
// H = N, so y_k = DFT_N(v_k)); the factor is a circular shift of the FFT
// input by A_k mod N, folded into the FIR's placement.
//
// Single pass (N <= 8192): one CTA per frame computes the FIR straight into
// shared memory, runs an in-place mixed-radix Stockham FFT there and writes
// the spectrum row and the tone channels.
//
// Two passes (N > 8192): the four-step split N = N1*N2 with input index
// p = N2*p1 + p2 and output index c = c1 + N1*c2,
//   Z[c1][p2]     = W_N^{p2*c1} * sum_{p1} v[N2*p1 + p2] W_{N1}^{p1*c1}   (pass A)
//   y[c1 + N1*c2] = sum_{p2} Z[c1][p2] W_{N2}^{p2*c2}                     (pass B)
// with W_L = exp(-2*pi*i/L).  When N2 is even and a pass-A CTA holds at
// least two transforms (the common case), the FIR runs first as its own
// coalesced kernel into V [frames][N] and pass A takes its N1 x GA points as
// 2-D TMA boxes of V; otherwise pass A computes the FIR of its points itself
// (input read in runs of GA samples).  Pass A: one CTA per (frame, GA
// consecutive p2): GA interleaved FFTs of length N1, the twiddle W_N^{p2*c1}
// (the product of three FP64-built entries, one per 8-bit digit of p2*c1,
// from tables in shared memory), Z stored in runs of GA points.  Pass B: one
// CTA per (frame, GB consecutive c1): GB rows of Z (one bulk copy when N2 is
// even), GB interleaved FFTs of length N2, the spectrum stored in runs of GB
// points, and the group's tones from a list built on the host.  V and Z hold
// a batch of frames (1 GB each) between the launches.
//
// Each sub-transform runs the fewest Stockham passes of radices up to 25:
// 16, 8, 4, 2 from fft_dev.cuh, 3, 5, 7 from their definitions, and the
// composites 6 ... 25 as register DFTs of two factors with their inner
// twiddles from a constant table.
// FFT stages follow the conventions of fft_dev.cuh (Stockham autosort,
// butterfly j reads x[j + r*n/R], twiddle W_{R*Ns}^{r*k} with k = j mod Ns,
// writes y[(j/Ns)*R*Ns + k + r*Ns]; twiddle table [(r-1)*Ns + k] per stage).
// Stages alternate between two shared-memory buffers of the G x n <= 4096
// (256-thread CTAs) or 8192 (512-thread CTAs) points (G transforms interleaved, element (i, g) at i*G + g, padded one
// element in 16).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "dev_common.cuh"
#include "fft_dev.cuh"
#include "rfr_internal.h"

namespace rfr {

namespace {

// Two CTA shapes: TH threads hold TH * 16 points (G * n): 256 threads with
// 4096 points (three CTAs per SM), or 512 threads with 8192 points (one CTA
// per SM, for the largest N, where 4096 points would force single-point runs).
constexpr int kGElemsMax = 8192;
template <int TH>
struct GenCfg {
    static constexpr int kElems = TH * 16;
    static constexpr int kMinBlocks = TH == 256 ? 3 : 1;
};
constexpr int kTwDigit = 256;                      // inter-pass twiddle tables: 3 x 256 entries
constexpr int kGMax = 64;                          // transforms interleaved per CTA

__device__ __forceinline__ int gpad(int e) { return e + (e >> 4); }

// cos(2*pi*j/R) and sin(2*pi*j/R) for R = 3, 5, 7 and 0 <= j < R.
template <int R>
__device__ __forceinline__ constexpr float cos_r(int j) {
    if (j == 0) return 1.0f;
    if (R == 3) return -0.5f;
    if (R == 5) return (j == 1 || j == 4) ? 0.30901699437494742f : -0.80901699437494742f;
    return (j == 1 || j == 6) ? 0.62348980185873353f
                              : ((j == 2 || j == 5) ? -0.22252093395631440f : -0.90096886790241913f);
}
template <int R>
__device__ __forceinline__ constexpr float sin_r(int j) {
    if (j == 0) return 0.0f;
    const float s = R == 3   ? 0.86602540378443865f
                    : R == 5 ? ((j == 1 || j == 4) ? 0.95105651629515357f : 0.58778525229247313f)
                             : ((j == 1 || j == 6) ? 0.78183148246802981f
                                                   : ((j == 2 || j == 5) ? 0.97492791218182361f : 0.43388373911755812f));
    return 2 * j < R ? s : -s;
}

// Length-R DFT for odd R (3, 5, 7) from the definition, pairing q with R-q:
//   y_k     = a_0 + sum_{q=1}^{(R-1)/2} [c_kq (a_q + a_{R-q}) - i s_kq (a_q - a_{R-q})]
//   y_{R-k} = the same with +i,
// c_j = cos(2*pi*j/R), s_j = sin(2*pi*j/R), indices mod R.
template <int R>
__device__ __forceinline__ void dft_odd(float2* x) {
    constexpr int H = (R - 1) / 2;
    float2 b[H], d[H];
    float2 y0 = x[0];
#pragma unroll
    for (int q = 1; q <= H; ++q) {
        b[q - 1] = cadd(x[q], x[R - q]);
        d[q - 1] = csub(x[q], x[R - q]);
        y0 = cadd(y0, b[q - 1]);
    }
    float2 out[R];
    out[0] = y0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        float tr = x[0].x, ti = x[0].y, ur = 0.f, ui = 0.f;
#pragma unroll
        for (int q = 1; q <= H; ++q) {
            const float c = cos_r<R>((k * q) % R), s = sin_r<R>((k * q) % R);
            tr = fmaf(c, b[q - 1].x, tr);
            ti = fmaf(c, b[q - 1].y, ti);
            ur = fmaf(s, d[q - 1].x, ur);
            ui = fmaf(s, d[q - 1].y, ui);
        }
        out[k] = make_float2(tr + ui, ti - ur);          // t - i*u
        out[R - k] = make_float2(tr - ui, ti + ur);      // t + i*u
    }
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = out[r];
}


// Inner twiddles of the composite radices (registers-only DFTs of R = A*B):
// exp(-2*pi*i*e/R) for e < R, FP64 cos/sin rounded to FP32, R in
// {6, 9, 10, 12, 15, 20, 25} back to back.
__constant__ float2 c_inner_tw[97] = {
    {1.0f, -0.0f}, {0.5f, -0.8660253882408142f}, {-0.5f, -0.8660253882408142f},
    {-1.0f, -1.2246468525851679e-16f}, {-0.5f, 0.8660253882408142f}, {0.5f, 0.8660253882408142f},
    {1.0f, -0.0f}, {0.7660444378852844f, -0.6427876353263855f}, {0.1736481785774231f, -0.9848077297210693f},
    {-0.5f, -0.8660253882408142f}, {-0.9396926164627075f, -0.3420201539993286f}, {-0.9396926164627075f, 0.3420201539993286f},
    {-0.5f, 0.8660253882408142f}, {0.1736481785774231f, 0.9848077297210693f}, {0.7660444378852844f, 0.6427876353263855f},
    {1.0f, -0.0f}, {0.80901700258255f, -0.5877852439880371f}, {0.30901700258255005f, -0.9510565400123596f},
    {-0.30901700258255005f, -0.9510565400123596f}, {-0.80901700258255f, -0.5877852439880371f}, {-1.0f, -1.2246468525851679e-16f},
    {-0.80901700258255f, 0.5877852439880371f}, {-0.30901700258255005f, 0.9510565400123596f}, {0.30901700258255005f, 0.9510565400123596f},
    {0.80901700258255f, 0.5877852439880371f}, {1.0f, -0.0f}, {0.8660253882408142f, -0.5f},
    {0.5f, -0.8660253882408142f}, {6.123234262925839e-17f, -1.0f}, {-0.5f, -0.8660253882408142f},
    {-0.8660253882408142f, -0.5f}, {-1.0f, -1.2246468525851679e-16f}, {-0.8660253882408142f, 0.5f},
    {-0.5f, 0.8660253882408142f}, {-1.8369701465288538e-16f, 1.0f}, {0.5f, 0.8660253882408142f},
    {0.8660253882408142f, 0.5f}, {1.0f, -0.0f}, {0.9135454297065735f, -0.4067366421222687f},
    {0.6691306233406067f, -0.7431448101997375f}, {0.30901700258255005f, -0.9510565400123596f}, {-0.10452846437692642f, -0.9945219159126282f},
    {-0.5f, -0.8660253882408142f}, {-0.80901700258255f, -0.5877852439880371f}, {-0.9781476259231567f, -0.2079116851091385f},
    {-0.9781476259231567f, 0.2079116851091385f}, {-0.80901700258255f, 0.5877852439880371f}, {-0.5f, 0.8660253882408142f},
    {-0.10452846437692642f, 0.9945219159126282f}, {0.30901700258255005f, 0.9510565400123596f}, {0.6691306233406067f, 0.7431448101997375f},
    {0.9135454297065735f, 0.4067366421222687f}, {1.0f, -0.0f}, {0.9510565400123596f, -0.30901700258255005f},
    {0.80901700258255f, -0.5877852439880371f}, {0.5877852439880371f, -0.80901700258255f}, {0.30901700258255005f, -0.9510565400123596f},
    {6.123234262925839e-17f, -1.0f}, {-0.30901700258255005f, -0.9510565400123596f}, {-0.5877852439880371f, -0.80901700258255f},
    {-0.80901700258255f, -0.5877852439880371f}, {-0.9510565400123596f, -0.30901700258255005f}, {-1.0f, -1.2246468525851679e-16f},
    {-0.9510565400123596f, 0.30901700258255005f}, {-0.80901700258255f, 0.5877852439880371f}, {-0.5877852439880371f, 0.80901700258255f},
    {-0.30901700258255005f, 0.9510565400123596f}, {-1.8369701465288538e-16f, 1.0f}, {0.30901700258255005f, 0.9510565400123596f},
    {0.5877852439880371f, 0.80901700258255f}, {0.80901700258255f, 0.5877852439880371f}, {0.9510565400123596f, 0.30901700258255005f},
    {1.0f, -0.0f}, {0.9685831665992737f, -0.24868988990783691f}, {0.8763066530227661f, -0.4817536771297455f},
    {0.728968620300293f, -0.6845471262931824f}, {0.5358268022537231f, -0.8443279266357422f}, {0.30901700258255005f, -0.9510565400123596f},
    {0.06279052048921585f, -0.9980267286300659f}, {-0.187381312251091f, -0.9822872281074524f}, {-0.4257792830467224f, -0.9048270583152771f},
    {-0.6374239921569824f, -0.7705132365226746f}, {-0.80901700258255f, -0.5877852439880371f}, {-0.9297764897346497f, -0.3681245446205139f},
    {-0.9921147227287292f, -0.12533323466777802f}, {-0.9921147227287292f, 0.12533323466777802f}, {-0.9297764897346497f, 0.3681245446205139f},
    {-0.80901700258255f, 0.5877852439880371f}, {-0.6374239921569824f, 0.7705132365226746f}, {-0.4257792830467224f, 0.9048270583152771f},
    {-0.187381312251091f, 0.9822872281074524f}, {0.06279052048921585f, 0.9980267286300659f}, {0.30901700258255005f, 0.9510565400123596f},
    {0.5358268022537231f, 0.8443279266357422f}, {0.728968620300293f, 0.6845471262931824f}, {0.8763066530227661f, 0.4817536771297455f},
    {0.9685831665992737f, 0.24868988990783691f}};

template <int R>
__host__ __device__ constexpr int inner_off() {
    if (R == 6) return 0;
    if (R == 9) return 6;
    if (R == 10) return 15;
    if (R == 12) return 25;
    if (R == 15) return 37;
    if (R == 20) return 52;
    if (R == 25) return 72;
    return -1;
}

// R = A*B with A the power-of-two part (when R has one and R/A > 1), else the
// smallest odd prime factor.
template <int R>
__host__ __device__ constexpr int split_a() {
    if (R % 16 == 0 && R > 16) return 16;
    if (R % 8 == 0 && R > 8) return 8;
    if (R % 4 == 0 && R > 4) return 4;
    if (R % 2 == 0 && R > 2) return 2;
    if (R % 3 == 0 && R > 3) return 3;
    if (R % 5 == 0 && R > 5) return 5;
    return 7;
}

// Length-R DFT in registers, natural order.  Composite R = A*B, input index
// n = n1 + A*n2 and output index k = B*k1 + k2:
//   X[B*k1 + k2] = sum_{n1} W_A^{n1*k1} W_R^{n1*k2} sum_{n2} x[n1 + A*n2] W_B^{n2*k2}.
template <int R>
__device__ __forceinline__ void dft_reg(float2* x) {
    if constexpr (R == 2 || R == 4 || R == 8 || R == 16) {
        dft_small<R>(x);
    } else if constexpr (R == 3 || R == 5 || R == 7) {
        dft_odd<R>(x);
    } else {
        constexpr int A = split_a<R>(), B = R / A;
        static_assert(inner_off<R>() >= 0, "composite radix without an inner twiddle table");
        float2 y[R];
#pragma unroll
        for (int n1 = 0; n1 < A; ++n1) {
            float2 t[B];
#pragma unroll
            for (int n2 = 0; n2 < B; ++n2) t[n2] = x[n1 + A * n2];
            dft_reg<B>(t);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2)
                y[n1 * B + k2] = (n1 == 0 || k2 == 0) ? t[k2] : cmul(t[k2], c_inner_tw[inner_off<R>() + n1 * k2]);
        }
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
            float2 t[A];
#pragma unroll
            for (int n1 = 0; n1 < A; ++n1) t[n1] = y[n1 * B + k2];
            dft_reg<A>(t);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) x[B * k1 + k2] = t[k1];
        }
    }
}

template <int R>
__device__ __forceinline__ void dft_any(float2* x) {
    dft_reg<R>(x);
}

// The R points x0 + r*s (r < R) of a padded buffer: when s is a multiple of
// 16, gpad(x0 + r*s) = gpad(x0) + r*(s + s/16) exactly, so one padded index
// and a constant step replace R of them.
template <int R>
__device__ __forceinline__ void load_strided(float2 (&v)[R], const float2* __restrict__ src, int x0, int s) {
    if ((s & 15) == 0) {
        const float2* p = src + gpad(x0);
        const int st = s + (s >> 4);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = p[r * st];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[gpad(x0 + r * s)];
    }
}
template <int R>
__device__ __forceinline__ void store_strided(const float2 (&v)[R], float2* __restrict__ dst, int x0, int s) {
    if ((s & 15) == 0) {
        float2* p = dst + gpad(x0);
        const int st = s + (s >> 4);
#pragma unroll
        for (int r = 0; r < R; ++r) p[r * st] = v[r];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) dst[gpad(x0 + r * s)] = v[r];
    }
}

// One Stockham stage of radix R over G = 2^gl2 interleaved transforms of
// length n, from src to dst (points at [gpad(i*G + g)]).
// j / Ns as umulhi(j, ns_magic) with ns_magic = ceil(2^32 / Ns) for Ns > 1:
// exact while j * Ns < 2^32 (here j, Ns < 2^13).
template <int R, int TH>
__device__ __forceinline__ void gen_stage(const float2* __restrict__ src, float2* __restrict__ dst, int n, int gl2,
                                          int Ns, uint32_t ns_magic, const float2* __restrict__ tw) {
    const int nR = n / R;
    const int nb = nR << gl2;
    const int gm = (1 << gl2) - 1;
#pragma unroll 2
    for (int u = threadIdx.x; u < nb; u += TH) {
        const int g = u & gm, j = u >> gl2;
        const int q = Ns == 1 ? j : static_cast<int>(__umulhi(static_cast<uint32_t>(j), ns_magic));
        const int k = j - q * Ns;
        float2 v[R];
        load_strided<R>(v, src, u, nb);                      // points (j + r*nR)*G + g
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(tw + (r - 1) * Ns + k));
        }
        dft_any<R>(v);
        const int base = (j - k) * R + k;
        store_strided<R>(v, dst, (base << gl2) + g, Ns << gl2);   // points (base + r*Ns)*G + g
    }
    __syncthreads();
}

// The last stage of a transform: the same butterflies, each output point
// handed to sink(e, value) (e = c*G + g: output c of transform g) instead of
// being written back to shared memory.
template <int R, int TH, typename Sink>
__device__ __forceinline__ void gen_stage_out(const float2* __restrict__ src, int n, int gl2, int Ns,
                                              uint32_t ns_magic, const float2* __restrict__ tw, Sink& sink) {
    const int nR = n / R;
    const int nb = nR << gl2;
    const int gm = (1 << gl2) - 1;
    for (int u = threadIdx.x; u < nb; u += TH) {
        const int g = u & gm, j = u >> gl2;
        const int q = Ns == 1 ? j : static_cast<int>(__umulhi(static_cast<uint32_t>(j), ns_magic));
        const int k = j - q * Ns;
        float2 v[R];
        load_strided<R>(v, src, u, nb);                      // points (j + r*nR)*G + g
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(tw + (r - 1) * Ns + k));
        }
        dft_any<R>(v);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) sink(((base + r * Ns) << gl2) + g, v[r]);
    }
}

// The whole transform with its output points delivered to `sink` by the
// last stage; the points start in buf0.  Returns the buffer the last stage
// did not read (free for the caller).
template <int TH, typename Sink>
__device__ float2* gen_fft_to(float2* buf0, float2* buf1, const GenFft& f, int gl2, const float2* __restrict__ tw,
                              Sink sink) {
    float2* src = buf0;
    float2* dst = buf1;
    for (int s = 0; s < f.nst; ++s) {
        const float2* t = tw + f.tw_off[s];
        const bool last = s == f.nst - 1;
#define RFR_GEN_CASE(RR)                                                                              \
    case RR:                                                                                          \
        if (last) gen_stage_out<RR, TH>(src, f.n, gl2, f.ns[s], f.ns_magic[s], t, sink);              \
        else gen_stage<RR, TH>(src, dst, f.n, gl2, f.ns[s], f.ns_magic[s], t);                        \
        break;
        switch (f.radix[s]) {
            RFR_GEN_CASE(16)
            RFR_GEN_CASE(25)
            RFR_GEN_CASE(20)
            RFR_GEN_CASE(15)
            RFR_GEN_CASE(12)
            RFR_GEN_CASE(10)
            RFR_GEN_CASE(9)
            RFR_GEN_CASE(8)
            RFR_GEN_CASE(7)
            RFR_GEN_CASE(6)
            RFR_GEN_CASE(5)
            RFR_GEN_CASE(4)
            RFR_GEN_CASE(3)
            RFR_GEN_CASE(2)
        default: break;
        }
#undef RFR_GEN_CASE
        if (!last) {
            float2* tmp = src;
            src = dst;
            dst = tmp;
        }
    }
    return dst;
}

// Compiled-in transform shapes (the four-step passes of N = 10^5 and 10^7): the same stages, loads, twiddles and butterflies as gen_fft_to in
// the same order (so the same results), with the length, the span, the
// group count and every stride known at compile time, so the index
// arithmetic folds into constants and immediate offsets.
template <int R, int TH, int N, int GL2, int NS, bool OUT, typename Sink>
__device__ __forceinline__ void fixed_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                            const float2* __restrict__ tw, Sink& sink) {
    constexpr int nb = (N / R) << GL2;
    constexpr int iters = (nb + TH - 1) / TH;
#pragma unroll
    for (int i = 0; i < iters; ++i) {
        const int u = static_cast<int>(threadIdx.x) + i * TH;
        if (nb % TH != 0 && u >= nb) break;
        const int g = u & ((1 << GL2) - 1), j = u >> GL2;
        const int k = NS == 1 ? 0 : j % NS;
        float2 v[R];
        load_strided<R>(v, src, u, nb);                      // points (j + r*nR)*G + g
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(tw + (r - 1) * NS + k));
        }
        dft_any<R>(v);
        const int base = (j - k) * R + k;
        if constexpr (OUT) {
#pragma unroll
            for (int r = 0; r < R; ++r) sink(((base + r * NS) << GL2) + g, v[r]);
        } else {
            store_strided<R>(v, dst, (base << GL2) + g, NS << GL2);
        }
    }
    if constexpr (!OUT) __syncthreads();
}

template <int TH, int GL2, int N, int NS, int R, int... Rest>
struct FixedFft {
    // stages from src; returns the buffer the last stage did not read
    template <typename Sink>
    __device__ __forceinline__ static float2* run(float2* src, float2* dst, const float2* __restrict__ tw, Sink& sink) {
        if constexpr (sizeof...(Rest) == 0) {
            fixed_stage<R, TH, N, GL2, NS, true>(src, dst, tw, sink);
            return dst;
        } else {
            fixed_stage<R, TH, N, GL2, NS, false>(src, dst, tw, sink);
            return FixedFft<TH, GL2, N, NS * R, Rest...>::run(dst, src, tw + (NS > 1 ? (R - 1) * NS : 0), sink);
        }
    }
};

// The compiled-in shapes: {id, threads, log2 of the transforms per CTA,
// length, radices}; ids 1.. as dispatched by fft_to below (a shape listed
// here for one pass is only taken by the pass that dispatches it).
struct FixedShape {
    int id, th, gl2, n, nst, radix[4];
};
constexpr FixedShape kFixedShapes[] = {
    {1, 256, 3, 400, 2, {25, 16, 0, 0}},     // N = 10^5, pass A
    {2, 256, 4, 250, 2, {25, 10, 0, 0}},     // N = 10^5, pass B
    {4, 512, 1, 3125, 3, {25, 25, 5, 0}},    // N = 10^7, pass A
    {5, 512, 1, 3200, 3, {25, 16, 8, 0}},    // N = 10^7, pass B
};

// gen_fft_to, through a compiled-in shape when `fix` names one (pass A
// dispatches its shape, pass B its own: more shapes in one kernel made its
// register allocation worse, with spills)
template <int TH, int PASS, typename Sink>
__device__ __forceinline__ float2* fft_to(float2* buf0, float2* buf1, const GenFft& f, int gl2,
                                          const float2* __restrict__ tw, int fix, Sink sink) {
    const float2* t0 = tw + f.tw_off[0];
    if constexpr (TH == 256 && PASS == 0) {
        if (fix == 1) return FixedFft<TH, 3, 400, 1, 25, 16>::run(buf0, buf1, t0, sink);
    } else if constexpr (TH == 256) {
        if (fix == 2) return FixedFft<TH, 4, 250, 1, 25, 10>::run(buf0, buf1, t0, sink);
    } else if constexpr (PASS == 0) {
        if (fix == 4) return FixedFft<TH, 1, 3125, 1, 25, 25, 5>::run(buf0, buf1, t0, sink);
    } else {
        if (fix == 5) return FixedFft<TH, 1, 3200, 1, 25, 16, 8>::run(buf0, buf1, t0, sink);
    }
    return gen_fft_to<TH>(buf0, buf1, f, gl2, tw, sink);
}

struct GenArgs {
    const uint32_t* carry;
    int64_t cl;
    const uint32_t* buf;
    int64_t F;              // frames in this launch
    int64_t k0;             // index of the launch's first frame within the push
    int N, T;
    int hop;                // samples between frames
    int gls;                // one-pass form: log2 of the frames per CTA iteration
    int64_t a0;             // absolute sample index of the virtual stream's first sample
    int sh_fixed;           // the frames' shift when hop == N (the same for all), else -1
    const float* h;         // [T*N]
    GenFft fa, fb;          // pass A (length N1) and pass B / single (length N2 = N)
    const float2* tw_a;
    const float2* tw_b;
    const float2* tw3;      // [3][256]: W_N^{i}, W_N^{256 i}, W_N^{65536 i}
    int N1, N2, gla, glb;
    uint32_t n2_magic;      // ceil(2^32 / N2): f / N2 = umulhi(f, n2_magic) for f < GB*N2
    float2* z;              // [F][N1][N2]
    const int32_t* bins;
    int n_tones;
    const int2* gtone;      // pass B: tones per group (see GenPlan)
    const int* goff;
    float2* full;
    int64_t full_ld;
    float2* tones;
    int64_t tones_ld;
    int64_t fo;             // frame offset in the caller's outputs
    int zbulk;              // pass B reads its Z rows by one bulk copy (16-byte aligned rows)
    int* status;            // device status word (bounded waits)
    // FIR ahead of pass A (see GenPlan::vtma): V [frames][N], and pass A's
    // boxes of it (vboxes boxes of vbox_rows rows x GA points, vsstride
    // points apart in shared memory)
    float2* v;
    int vtma, vbox_rows, vboxes, vsstride;
    int fixa, fixb;         // compiled-in shapes of pass A / B (kFixedShapes ids), 0: generic stages
};

// FIR of the points e = tid, tid + TH, ... < E of one frame into sm: point e
// sits at frame position pos(e) (or is zero when pos(e) < 0), eight points
// at a time.  A frame whose window lies entirely in the new buffer (the common
// case) reads it through one pointer; a frame that starts in the carry takes
// the per-sample carry / buffer select.
template <int TH, typename Pos>
__device__ __forceinline__ void fir_points(const GenArgs& a, int64_t base, int E, Pos pos_of, float2* sm) {
    constexpr int P = 8;
    const bool fast = base >= a.cl;
    for (int e0 = threadIdx.x; e0 < E; e0 += P * TH) {
        int pos[P];
        bool valid[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int e = e0 + q * TH;
            const int pp = e < E ? pos_of(e) : -1;
            valid[q] = pp >= 0;
            pos[q] = valid[q] ? pp : 0;        // an in-bounds dummy point, zeroed below
        }
        float ar[P], ai[P];
#pragma unroll
        for (int q = 0; q < P; ++q) ar[q] = ai[q] = 0.f;
        if (fast) {
            const float* hp = a.h;
            const uint32_t* xp = a.buf + (base - a.cl);
#pragma unroll 4
            for (int t = 0; t < a.T; ++t) {
                float hv[P];
                uint32_t xw[P];
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    hv[q] = __ldg(hp + pos[q]);
                    xw[q] = __ldg(xp + pos[q]);
                }
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const float2 x = iq_to_f2(xw[q]);
                    ar[q] = fmaf(hv[q], x.x, ar[q]);
                    ai[q] = fmaf(hv[q], x.y, ai[q]);
                }
                hp += a.N;
                xp += a.N;
            }
        } else {
            for (int t = 0; t < a.T; ++t) {
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int64_t o = static_cast<int64_t>(t) * a.N + pos[q];
                    const int64_t vi = base + o;
                    const float hv = __ldg(a.h + o);
                    const float2 x = iq_to_f2(vi < a.cl ? __ldg(a.carry + vi) : __ldg(a.buf + (vi - a.cl)));
                    ar[q] = fmaf(hv, x.x, ar[q]);
                    ai[q] = fmaf(hv, x.y, ai[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int e = e0 + q * TH;
            if (e < E) sm[gpad(e)] = valid[q] ? make_float2(ar[q], ai[q]) : make_float2(0.f, 0.f);
        }
    }
}

// Frames keep the phase of the absolute time origin: the FFT input index q
// holds the window position (q - s) mod N, s = (absolute index of the
// window's first sample) mod N, so that channel c is the stream mixed down by
// exp(-2*pi*i*c*m/N) for every hop (s = 0 whenever the hop is N).
__device__ __forceinline__ int frame_shift(const GenArgs& a, int64_t base) {
    if (a.sh_fixed >= 0) return a.sh_fixed;
    const int64_t s = (a.a0 + base) % a.N;
    return static_cast<int>(s < 0 ? s + a.N : s);
}

// Shared memory: two buffers of gpad(elems) points each.
__device__ __forceinline__ float2* second_buffer(float2* sm, int elems) { return sm + gpad(elems) + 1; }

// FIR of G = 2^gls consecutive frames (the first at stream position base0,
// frame g at base0 + g*hop with shift shs[g]) into sm, interleaved: point e =
// i*G + g is FFT input i of frame g; frames g >= nf are zero.  Eight points
// at a time per thread, taps summed as in fir_points.
template <int TH>
__device__ __forceinline__ void fir_frames(const GenArgs& a, int64_t base0, int E, int gls, int nf,
                                           const int* shs, float2* sm) {
    constexpr int P = 8;
    const int G = 1 << gls, N = a.N;
    const bool fast = base0 >= a.cl;
    for (int e0 = threadIdx.x; e0 < E; e0 += P * TH) {
        int hoff[P], xoff[P];
        bool valid[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int e = e0 + q * TH;
            const int g = e & (G - 1), i = e >> gls;
            valid[q] = e < E && g < nf;
            const int sh = valid[q] ? shs[g] : 0;
            const int pos = i >= sh ? i - sh : i - sh + N;
            hoff[q] = valid[q] ? pos : 0;                     // in-bounds dummy, zeroed below
            xoff[q] = valid[q] ? g * a.hop + pos : 0;
        }
        float ar[P], ai[P];
#pragma unroll
        for (int q = 0; q < P; ++q) ar[q] = ai[q] = 0.f;
        if (fast) {
            const float* hp = a.h;
            const uint32_t* xp = a.buf + (base0 - a.cl);
#pragma unroll 4
            for (int t = 0; t < a.T; ++t) {
                float hv[P];
                uint32_t xw[P];
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    hv[q] = __ldg(hp + hoff[q]);
                    xw[q] = __ldg(xp + xoff[q]);
                }
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const float2 x = iq_to_f2(xw[q]);
                    ar[q] = fmaf(hv[q], x.x, ar[q]);
                    ai[q] = fmaf(hv[q], x.y, ai[q]);
                }
                hp += N;
                xp += N;
            }
        } else {
            for (int t = 0; t < a.T; ++t) {
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const float hv = __ldg(a.h + static_cast<int64_t>(t) * N + hoff[q]);
                    const int64_t vi = base0 + static_cast<int64_t>(t) * N + xoff[q];
                    const float2 x = iq_to_f2(vi < a.cl ? __ldg(a.carry + vi) : __ldg(a.buf + (vi - a.cl)));
                    ar[q] = fmaf(hv, x.x, ar[q]);
                    ai[q] = fmaf(hv, x.y, ai[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int e = e0 + q * TH;
            if (e < E) sm[gpad(e)] = valid[q] ? make_float2(ar[q], ai[q]) : make_float2(0.f, 0.f);
        }
    }
}

// One pass (N <= 8192): G = 2^gls consecutive frames per CTA iteration,
// interleaved (point i of frame g at i*G + g), so that a small N still gives
// every thread of the CTA butterflies in each stage.
template <int TH>
__global__ void __launch_bounds__(TH, GenCfg<TH>::kMinBlocks) gen_single_kernel(const GenArgs a) {
    extern __shared__ float2 sm[];
    const int gls = a.gls, G = 1 << gls, N = a.N;
    const int E = N << gls;
    float2* sm1 = second_buffer(sm, E);
    int* shs = reinterpret_cast<int*>(sm + 2 * (gpad(E) + 1));    // the G frames' shifts
    const int64_t iters = (a.F + G - 1) >> gls;
    for (int64_t it = blockIdx.x; it < iters; it += gridDim.x) {
        const int64_t kk0 = it << gls;
        const int nf = a.F - kk0 < G ? static_cast<int>(a.F - kk0) : G;
        const int64_t k0 = a.k0 + kk0;                       // the first frame's index in the push
        if (static_cast<int>(threadIdx.x) < G) shs[threadIdx.x] = frame_shift(a, (k0 + threadIdx.x) * a.hop);
        __syncthreads();
        if (gls == 0) {
            const int sh = shs[0];
            fir_points<TH>(a, k0 * a.hop, N, [=](int e) { return e >= sh ? e - sh : e - sh + N; }, sm);
        } else {
            fir_frames<TH>(a, k0 * a.hop, E, gls, nf, shs, sm);
        }
        __syncthreads();
        float2* rows = a.full ? a.full + (a.fo + k0) * a.full_ld : nullptr;
        const int64_t ld = a.full_ld;
        const bool keep = a.n_tones > 0;
        float2* const freebuf = (a.fb.nst & 1) ? sm1 : sm;   // the buffer the last stage does not read
        // the last stage writes the spectrum rows and, for the tone gather, a
        // copy into the free shared-memory buffer
        gen_fft_to<TH>(sm, sm1, a.fb, gls, a.tw_b, [=](int e, float2 v) {
            const int g = e & (G - 1);
            if (rows && g < nf) rows[g * ld + (e >> gls)] = v;
            if (keep) freebuf[gpad(e)] = v;
        });
        if (keep) {
            __syncthreads();
            for (int i = threadIdx.x; i < (a.n_tones << gls); i += TH) {
                const int t = i >> gls, g = i & (G - 1);
                if (g < nf) a.tones[t * a.tones_ld + a.fo + k0 + g] = freebuf[gpad((__ldg(a.bins + t) << gls) + g)];
            }
        }
        __syncthreads();
    }
}

// The FIR of the two-pass form ahead of pass A: v[k][q] for the launch's
// frames k and every FFT input index q (window position (q - s) mod N), into
// V in natural order.  One CTA per (frame, kFirThreads * kFirPts points),
// the frames of a point range consecutive in launch order (their windows
// overlap, and the range's taps are shared); consecutive threads take
// consecutive points, so every load and store is coalesced, and the small
// register footprint leaves many warps in flight.
// Taps are summed in the same order as fir_points (t = 0.. T-1 from zero).
constexpr int kFirThreads = 256, kFirPts = 8;
// TC > 0: T == TC known at compile time, so every load of a thread (2 TC
// kFirPts) is issued before the first use; TC == 0: any T.
template <int TC>
__global__ void __launch_bounds__(kFirThreads) gen_fir_kernel(const GenArgs a) {
    const int64_t kk = blockIdx.x;
    const int64_t base = (a.k0 + kk) * a.hop;
    const int sh = frame_shift(a, base);
    const int N = a.N;
    const int T = TC > 0 ? TC : a.T;
    const int qb = static_cast<int>(blockIdx.y) * (kFirThreads * kFirPts) + static_cast<int>(threadIdx.x);
    int pos[kFirPts];
    float ar[kFirPts], ai[kFirPts];
#pragma unroll
    for (int j = 0; j < kFirPts; ++j) {
        const int q = qb + j * kFirThreads;
        pos[j] = q < N ? (q >= sh ? q - sh : q - sh + N) : 0;
        ar[j] = ai[j] = 0.f;
    }
    if (base >= a.cl) {
        const uint32_t* xp = a.buf + (base - a.cl);
        if constexpr (TC > 0) {
            float hv[TC][kFirPts];
            uint32_t xw[TC][kFirPts];
#pragma unroll
            for (int t = 0; t < TC; ++t)
#pragma unroll
                for (int j = 0; j < kFirPts; ++j) {
                    hv[t][j] = __ldg(a.h + (t * N + pos[j]));
                    xw[t][j] = __ldg(xp + (t * N + pos[j]));
                }
#pragma unroll
            for (int t = 0; t < TC; ++t)
#pragma unroll
                for (int j = 0; j < kFirPts; ++j) {
                    const float2 x = iq_to_f2(xw[t][j]);
                    ar[j] = fmaf(hv[t][j], x.x, ar[j]);
                    ai[j] = fmaf(hv[t][j], x.y, ai[j]);
                }
        } else {
            for (int t = 0; t < T; ++t) {
#pragma unroll
                for (int j = 0; j < kFirPts; ++j) {
                    const float hv = __ldg(a.h + (t * N + pos[j]));
                    const float2 x = iq_to_f2(__ldg(xp + (t * N + pos[j])));
                    ar[j] = fmaf(hv, x.x, ar[j]);
                    ai[j] = fmaf(hv, x.y, ai[j]);
                }
            }
        }
    } else {
        for (int t = 0; t < T; ++t) {
#pragma unroll
            for (int j = 0; j < kFirPts; ++j) {
                const int64_t o = static_cast<int64_t>(t) * N + pos[j];
                const int64_t vi = base + o;
                const float hv = __ldg(a.h + o);
                const float2 x = iq_to_f2(vi < a.cl ? __ldg(a.carry + vi) : __ldg(a.buf + (vi - a.cl)));
                ar[j] = fmaf(hv, x.x, ar[j]);
                ai[j] = fmaf(hv, x.y, ai[j]);
            }
        }
    }
    float2* vrow = a.v + kk * N;
#pragma unroll
    for (int j = 0; j < kFirPts; ++j) {
        const int q = qb + j * kFirThreads;
        if (q < N) vrow[q] = make_float2(ar[j], ai[j]);
    }
}

// The FIR ahead of pass A for hop == N (every frame shifted alike): a thread
// takes kMfPts points of kMfFrames consecutive frames.  Frame f + g reads
// input blocks g .. g + T - 1 (block r = samples base + r*N + pos), so the
// kMfFrames + T - 1 blocks are loaded and converted once and each feeds the
// frames that use it, in tap order t = r - g = 0 .. T-1 from zero (the same
// sums as gen_fir_kernel, bit for bit); the taps are loaded once for all the
// thread's frames.
constexpr int kMfPts = 4, kMfFrames = 4;
template <int TC>
__global__ void __launch_bounds__(kFirThreads) gen_fir_frames_kernel(const GenArgs a) {
    constexpr int G = kMfFrames, P = kMfPts, R = G + TC - 1;
    const int64_t f0 = static_cast<int64_t>(blockIdx.x) * G;            // first frame (of this launch)
    const int gn = static_cast<int>(a.F - f0 < G ? a.F - f0 : G);       // frames of this row that exist
    const int64_t base = (a.k0 + f0) * a.hop;
    const int N = a.N, sh = a.sh_fixed;
    const int qb = static_cast<int>(blockIdx.y) * (kFirThreads * P) + static_cast<int>(threadIdx.x);
    int pos[P];
    float hv[TC][P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int q = qb + j * kFirThreads;
        pos[j] = q < N ? (q >= sh ? q - sh : q - sh + N) : 0;
#pragma unroll
        for (int t = 0; t < TC; ++t) hv[t][j] = __ldg(a.h + (t * N + pos[j]));
    }
    float ar[G][P], ai[G][P];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int j = 0; j < P; ++j) ar[g][j] = ai[g][j] = 0.f;
    const bool fast = base >= a.cl;
    const uint32_t* xp = a.buf + (base - a.cl);
    // every block's loads issued before the first use (blocks past the last
    // frame of the row read as zero and feed no existing frame)
    uint32_t w[R][P];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int64_t o = static_cast<int64_t>(r) * N + pos[j];
            if (r >= gn + TC - 1) w[r][j] = 0u;
            else if (fast) w[r][j] = __ldg(xp + o);
            else w[r][j] = base + o < a.cl ? __ldg(a.carry + (base + o)) : __ldg(a.buf + (base + o - a.cl));
        }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float2 x[P];
#pragma unroll
        for (int j = 0; j < P; ++j) x[j] = iq_to_f2(w[r][j]);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int t = r - g;
            if (t < 0 || t >= TC) continue;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                ar[g][j] = fmaf(hv[t][j], x[j].x, ar[g][j]);
                ai[g][j] = fmaf(hv[t][j], x[j].y, ai[g][j]);
            }
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (g >= gn) break;
        float2* vrow = a.v + (f0 + g) * N;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int q = qb + j * kFirThreads;
            if (q < N) vrow[q] = make_float2(ar[g][j], ai[g][j]);
        }
    }
}

template <int TH>
__global__ void __launch_bounds__(TH, GenCfg<TH>::kMinBlocks)
    gen_pass_a_kernel(const GenArgs a, const __grid_constant__ CUtensorMap tmv) {
    extern __shared__ float2 sm[];
    const int GA = 1 << a.gla;
    const int groups = (a.N2 + GA - 1) >> a.gla;
    const int E = a.N1 << a.gla;
    float2* sm1 = second_buffer(sm, E);
    // the digit tables of W_N^m, m = a*65536 + b*256 + c (N <= 2^24)
    float2* stw = sm + 2 * (gpad(E) + 1);
    for (int i = threadIdx.x; i < 3 * kTwDigit; i += TH) stw[i] = __ldg(a.tw3 + i);
    // V's boxes land 128-byte aligned in the second buffer; mbarrier after the tables
    float2* vst = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(sm1) + 127) & ~uintptr_t(127));
    uint64_t* vbar = reinterpret_cast<uint64_t*>(stw + 3 * kTwDigit);
    if (a.vtma && threadIdx.x == 0) {
        mbar_init(vbar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t vphase = 0;
    for (int64_t it = blockIdx.x; it < a.F * groups; it += gridDim.x) {
        const int64_t kk = it / groups;
        const int g0 = static_cast<int>(it - kk * groups) << a.gla;
        const int N2 = a.N2, gla = a.gla;
        if (a.vtma) {
            // points p1*GA + g = V[kk][p1*N2 + g0 + g]: boxes of rows of V
            // viewed as [frames*N1][N2] (columns past N2 read as zero)
            if (threadIdx.x == 0) {
                mbar_arrive_expect_tx(vbar, static_cast<uint32_t>(a.vboxes * a.vbox_rows * GA * 8));
                for (int b = 0; b < a.vboxes; ++b)
                    tma_load_2d(vst + b * a.vsstride, &tmv, g0,
                                static_cast<int32_t>(kk * a.N1 + b * a.vbox_rows), vbar);
            }
            if (!mbar_wait(vbar, vphase, a.status)) return;
            vphase ^= 1u;
            for (int b = 0; b < a.vboxes; ++b) {
                const int rows = min(a.vbox_rows, a.N1 - b * a.vbox_rows);
                const int o = b * a.vbox_rows * GA;
                for (int e = threadIdx.x; e < rows * GA; e += TH) sm[gpad(o + e)] = vst[b * a.vsstride + e];
            }
        } else {
            const int64_t base = (a.k0 + kk) * a.hop;
            const int sh = frame_shift(a, base);
            const int N = a.N;
            fir_points<TH>(a, base, E,
                       [=](int e) {
                           const int g = e & (GA - 1);
                           if (g0 + g >= N2) return -1;
                           const int q = (e >> gla) * N2 + g0 + g;          // FFT input index
                           return q >= sh ? q - sh : q - sh + N;            // window position
                       },
                       sm);
        }
        __syncthreads();
        // the last stage multiplies by W_N^{p2*c1} and stores Z directly
        float2* zf = a.z + kk * a.N;
        fft_to<TH, 0>(sm, sm1, a.fa, a.gla, a.tw_a, a.fixa, [=](int e, float2 v) {
            const int g = e & (GA - 1), c1 = e >> gla, p2 = g0 + g;
            if (p2 < N2) {
                const int m = p2 * c1;                       // < N1*N2 = N
                const float2 w = cmul(cmul(stw[m & 255], stw[kTwDigit + ((m >> 8) & 255)]), stw[2 * kTwDigit + (m >> 16)]);
                zf[static_cast<int64_t>(c1) * N2 + p2] = cmul(v, w);
            }
        });
        fence_proxy_async_smem();   // shared-memory reads done before the next box lands
        __syncthreads();
    }
}

template <int TH>
__global__ void __launch_bounds__(TH, GenCfg<TH>::kMinBlocks) gen_pass_b_kernel(const GenArgs a) {
    extern __shared__ float2 sm[];
    const int GB = 1 << a.glb;
    const int groups = (a.N1 + GB - 1) >> a.glb;
    const int E = a.N2 << a.glb;
    float2* sm1 = second_buffer(sm, E);
    // the bulk copy lands 16-byte aligned in the second buffer (one spare
    // element at its end); its mbarrier follows the two buffers
    float2* zst = sm1 + ((reinterpret_cast<uintptr_t>(sm1) & 8) ? 1 : 0);
    uint64_t* zbar = reinterpret_cast<uint64_t*>(sm + 2 * (gpad(E) + 1));
    if (a.zbulk && threadIdx.x == 0) {
        mbar_init(zbar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t zphase = 0;
    for (int64_t it = blockIdx.x; it < a.F * groups; it += gridDim.x) {
        const int64_t kk = it / groups;
        const int c0 = static_cast<int>(it - kk * groups) << a.glb;
        // rows c0 .. c0+GB-1 of Z are one contiguous block of GB*N2 points
        const float2* zf = a.z + kk * a.N + static_cast<int64_t>(c0) * a.N2;
        const int rows = min(GB, a.N1 - c0);
        const int cnt = rows * a.N2;
        if (a.zbulk) {
            if (threadIdx.x == 0) {
                mbar_arrive_expect_tx(zbar, static_cast<uint32_t>(cnt) * 8u);
                tma_bulk_g2s(zst, zf, static_cast<uint32_t>(cnt) * 8u, zbar);
            }
            if (!mbar_wait(zbar, zphase, a.status)) return;
            zphase ^= 1u;
        }
#pragma unroll 4
        for (int f = threadIdx.x; f < E; f += TH) {
            const int g = static_cast<int>(__umulhi(static_cast<uint32_t>(f), a.n2_magic));   // f / N2
            const int p2 = f - g * a.N2;
            sm[gpad((p2 << a.glb) + g)] = f < cnt ? (a.zbulk ? zst[f] : zf[f]) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const int64_t k = a.k0 + kk;
        // the last stage stores the spectrum (runs of GB points) and, for the
        // tone gather, a copy in the free shared-memory buffer
        float2* row = a.full ? a.full + (a.fo + k) * a.full_ld : nullptr;
        const bool keep = a.n_tones > 0;
        float2* const freebuf = (a.fb.nst & 1) ? sm1 : sm;
        const int glb = a.glb, N1 = a.N1;
        fft_to<TH, 1>(sm, sm1, a.fb, a.glb, a.tw_b, a.fixb, [=](int e, float2 v) {
            const int g = e & (GB - 1), c2 = e >> glb;
            if (row && c0 + g < N1) row[c0 + g + static_cast<int64_t>(N1) * c2] = v;
            if (keep) freebuf[gpad(e)] = v;
        });
        if (keep) {
            __syncthreads();
            const int gi = c0 >> a.glb;
            const int i1 = __ldg(a.goff + gi + 1);
            for (int i = __ldg(a.goff + gi) + threadIdx.x; i < i1; i += TH) {
                const int2 te = __ldg(a.gtone + i);
                a.tones[te.x * a.tones_ld + a.fo + k] = freebuf[gpad(te.y)];
            }
        }
        fence_proxy_async_smem();   // shared-memory reads done before the next bulk copy writes
        __syncthreads();
    }
}

// ---------------------------------------------------------------- host side
bool smooth7(int64_t n) {
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

int floor_log2(int v) {
    int l = 0;
    while ((2 << l) <= v) ++l;
    return l;
}

// Radices of a length-n transform (the fewest passes of register DFTs),
// stage spans and twiddle-table offsets; appends the FP64-built twiddles to
// `tw` (offsets are absolute positions in `tw`).
bool build_fft(int n, GenFft* f, std::vector<float2>& tw, int rmax) {
    *f = GenFft{};
    f->n = n;
    int m = n, ns = 1;
    auto add = [&](int r) {
        if (f->nst >= kGenMaxStages) return false;
        f->radix[f->nst] = r;
        f->ns[f->nst] = ns;
        f->ns_magic[f->nst] = ns > 1 ? static_cast<uint32_t>(((uint64_t(1) << 32) + ns - 1) / ns) : 0u;
        f->tw_off[f->nst] = static_cast<int>(tw.size());
        if (ns > 1) {
            for (int rr = 1; rr < r; ++rr)
                for (int k = 0; k < ns; ++k) {
                    const int64_t e = static_cast<int64_t>(rr) * k, L = static_cast<int64_t>(r) * ns;
                    const double a = -2.0 * 3.14159265358979323846 * static_cast<double>(e % L) / static_cast<double>(L);
                    tw.push_back(make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a))));
                }
        }
        ++f->nst;
        ns *= r;
        return true;
    };
    // fewest passes: the largest radix of the register DFTs that divides
    // what is left (16 = 2^4 and the composites up to 25), at most rmax
    // (primes up to 7 always allowed).  Fewer passes measured faster than
    // smaller radices that keep every thread of the CTA busy.
    while (m > 1) {
        int r = 0;
        for (int c : {25, 20, 16, 15, 12, 10, 9, 8, 7, 6, 5, 4, 3, 2})
            if (m % c == 0 && (c <= rmax || c <= 7)) {
                r = c;
                break;
            }
        if (r == 0 || !add(r)) return false;
        m /= r;
    }
    return m == 1;
}

}  // namespace

bool gen_supported(int64_t n) { return n >= 2 && n <= (int64_t(1) << 24) && smooth7(n); }

cudaError_t gen_plan_set_tones(GenPlan* g, const int32_t* bins, int n_tones) {
    if (g->N1 <= 1 || n_tones <= 0) return cudaSuccess;
    const int gb = 1 << g->glb;
    const int groups = (g->N1 + gb - 1) / gb;
    std::vector<int> off(groups + 1, 0);
    for (int t = 0; t < n_tones; ++t) ++off[(bins[t] % g->N1) / gb + 1];
    for (int i = 0; i < groups; ++i) off[i + 1] += off[i];
    std::vector<int2> list(n_tones);
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (int t = 0; t < n_tones; ++t) {
        const int c1 = bins[t] % g->N1, c2 = bins[t] / g->N1, gi = c1 / gb;
        list[fill[gi]++] = make_int2(t, (c2 << g->glb) + c1 - gi * gb);
    }
    cudaError_t e;
    if ((e = cudaMalloc(&g->d_gtone, list.size() * sizeof(int2))) != cudaSuccess ||
        (e = cudaMalloc(&g->d_goff, off.size() * sizeof(int))) != cudaSuccess ||
        (e = cudaMemcpy(g->d_gtone, list.data(), list.size() * sizeof(int2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(g->d_goff, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

void gen_plan_free(GenPlan* g) {
    for (void* q : {static_cast<void*>(g->d_tw), static_cast<void*>(g->d_tw3),
                    static_cast<void*>(g->d_z), static_cast<void*>(g->d_gtone), static_cast<void*>(g->d_goff),
                    static_cast<void*>(g->d_v)})
        if (q) cudaFree(q);
    *g = GenPlan{};
}

cudaError_t gen_plan_reserve(GenPlan* g, int64_t frames) {
    if (g->N1 <= 1) return cudaSuccess;                       // one pass: no Z
    const int64_t want = std::max<int64_t>(1, std::min<int64_t>(frames, g->z_cap_frames));
    if (want <= g->z_frames) return cudaSuccess;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    if (g->d_z) cudaFree(g->d_z);
    if (g->d_v) cudaFree(g->d_v);
    g->d_z = g->d_v = nullptr;
    g->z_frames = 0;
    if ((e = cudaMalloc(&g->d_z, static_cast<size_t>(want) * g->N * 8)) != cudaSuccess) return e;
    if (g->vtma && (e = cudaMalloc(&g->d_v, static_cast<size_t>(want) * g->N * 8)) != cudaSuccess) return e;
    g->z_frames = want;
    return cudaSuccess;
}

cudaError_t gen_plan_init(GenPlan* g, int N, int64_t z_budget_bytes) {
    *g = GenPlan{};
    if (!gen_supported(N)) return cudaErrorInvalidValue;
    g->N = N;
    std::vector<float2> tw;
    // the best N = N1*N2 split for CTAs of `elems` points: largest
    // min(GA, GB) (the longest contiguous runs), then the more balanced, then
    // an even N2 (16-byte aligned rows: V and Z move by TMA)
    auto best_split = [&](int elems, int* n1o, int* n2o, int* score_o) {
        int best = -1, best_score = -1, best_bal = 0, best_even = 0;
        for (int n2 = 2; n2 <= elems; ++n2) {
            if (N % n2 != 0) continue;
            const int n1 = N / n2;
            if (n1 < 2 || n1 > elems) continue;
            const int ga = std::min(kGMax, 1 << floor_log2(elems / n1));
            const int gb = std::min(kGMax, 1 << floor_log2(elems / n2));
            const int score = std::min(ga, gb), bal = -std::abs(n1 - n2), even = n2 % 2 == 0;
            if (score > best_score || (score == best_score && bal > best_bal) ||
                (score == best_score && bal == best_bal && even > best_even)) {
                best = n2;
                best_score = score;
                best_bal = bal;
                best_even = even;
            }
        }
        *n2o = best;
        *n1o = best > 0 ? N / best : 0;
        *score_o = best_score;
        return best > 0;
    };
    if (N <= kGElemsMax) {
        g->threads = N <= GenCfg<256>::kElems ? 256 : 512;
        g->N1 = 1;
        g->N2 = N;
        // frames per CTA iteration: as many as fill the CTA's points (<= 64)
        g->gls = floor_log2(std::min(kGMax, g->threads * 16 / N));
        if (!build_fft(N, &g->fb, tw, 25)) return cudaErrorInvalidValue;
    } else {
        int n1 = 0, n2 = 0, score = 0;
        g->threads = 256;
        if (!best_split(GenCfg<256>::kElems, &n1, &n2, &score) || score < 4) {
            g->threads = 512;
            if (!best_split(GenCfg<512>::kElems, &n1, &n2, &score)) return cudaErrorInvalidValue;
        }
        const int elems = g->threads * 16;
        g->N1 = n1;
        g->N2 = n2;
        g->gla = floor_log2(std::min(kGMax, 1 << floor_log2(elems / g->N1)));
        g->glb = floor_log2(std::min(kGMax, 1 << floor_log2(elems / g->N2)));
        if (!build_fft(g->N1, &g->fa, tw, 25)) return cudaErrorInvalidValue;
        if (!build_fft(g->N2, &g->fb, tw, 25)) return cudaErrorInvalidValue;
    }
    cudaError_t e;
    const size_t twn = std::max<size_t>(tw.size(), 1);
    if ((e = cudaMalloc(&g->d_tw, twn * sizeof(float2))) != cudaSuccess) return e;
    if (!tw.empty() &&
        (e = cudaMemcpy(g->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    if (g->N1 > 1) {
        std::vector<float2> t3(3 * kTwDigit);
        auto w = [&](int64_t m) {
            const double a = -2.0 * 3.14159265358979323846 * static_cast<double>(m % N) / static_cast<double>(N);
            return make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
        };
        for (int i = 0; i < kTwDigit; ++i) {
            t3[i] = w(i);
            t3[kTwDigit + i] = w(static_cast<int64_t>(i) << 8);
            t3[2 * kTwDigit + i] = w(static_cast<int64_t>(i) << 16);
        }
        if ((e = cudaMalloc(&g->d_tw3, t3.size() * sizeof(float2))) != cudaSuccess ||
            (e = cudaMemcpy(g->d_tw3, t3.data(), t3.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        // Z (and V) are allocated by gen_plan_reserve, sized by the pushes (up to the budget)
        g->z_cap_frames = std::max<int64_t>(1, z_budget_bytes / (static_cast<int64_t>(N) * 8));
        // V by 2-D TMA: rows of N2 points (8 bytes each) need a 16-byte
        // multiple as pitch, and each box's first column g0 (a multiple of
        // GA) a 16-byte offset, so GA >= 2; pass A's N1 x GA points come in
        // boxes of at most 256 rows, each box 128-byte aligned in the second
        // buffer
        const int ga = 1 << g->gla;
        const int elems = g->N1 * ga;
        const int nb = (g->N1 + 255) / 256, rows = (g->N1 + nb - 1) / nb;
        const int sstride = (rows * ga + 15) / 16 * 16;
        if (g->N2 % 2 == 0 && ga >= 2 && tmap_encode_tiled_fn() != nullptr &&
            (nb - 1) * sstride + rows * ga + 16 <= elems + elems / 16 + 1) {
            g->vtma = 1;
            g->vboxes = nb;
            g->vbox_rows = rows;
            g->vsstride = sstride;
        }
    }
    return cudaSuccess;
}

namespace {
size_t smem_bytes(int elems) { return static_cast<size_t>(2 * (elems + elems / 16 + 1)) * sizeof(float2); }

template <int TH, typename K, typename... Args>
cudaError_t launch_gen(K kernel, int64_t items, int elems, int n_sms, cudaStream_t st, size_t extra_smem,
                       const Args&... args) {
    const size_t smem = smem_bytes(elems) + extra_smem;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, TH, smem) != cudaSuccess || occ < 1)
        occ = 1;
    const int64_t grid = std::min<int64_t>(items, static_cast<int64_t>(n_sms) * occ);
    kernel<<<static_cast<unsigned>(grid), TH, smem, st>>>(args...);
    return cudaGetLastError();
}
}  // namespace

namespace {
template <int TH>
cudaError_t gen_run(GenArgs a, const PfbLaunch& L, const GenPlan& g, cudaStream_t st) {
    if (g.N1 == 1) {
        a.F = L.F;
        a.k0 = 0;
        return launch_gen<TH>(gen_single_kernel<TH>, (L.F + (1 << g.gls) - 1) >> g.gls, g.N << g.gls, L.n_sms, st,
                              (size_t(1) << g.gls) * sizeof(int), a);
    }
    if (g.z_frames < 1 || !g.d_z) return cudaErrorInvalidValue;   // gen_plan_reserve first
    const int ga = 1 << g.gla, gb = 1 << g.glb;
    const int64_t groups_a = (g.N2 + ga - 1) / ga, groups_b = (g.N1 + gb - 1) / gb;
    // V as [z_frames * N1 rows][N2 points] of 8-byte elements, box GA x vbox_rows
    CUtensorMap tmv;
    std::memset(&tmv, 0, sizeof tmv);
    if (a.vtma) {
        if (!g.d_v) return cudaErrorInvalidValue;
        auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tmap_encode_tiled_fn());
        cuuint64_t dims[2] = {static_cast<cuuint64_t>(g.N2), static_cast<cuuint64_t>(g.z_frames) * g.N1};
        cuuint64_t strides[1] = {static_cast<cuuint64_t>(g.N2) * 8};
        cuuint32_t box[2] = {static_cast<cuuint32_t>(ga), static_cast<cuuint32_t>(g.vbox_rows)};
        cuuint32_t estr[2] = {1, 1};
        if (!enc || enc(&tmv, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, g.d_v, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    for (int64_t k0 = 0; k0 < L.F; k0 += g.z_frames) {
        a.k0 = k0;
        a.F = std::min<int64_t>(g.z_frames, L.F - k0);
        cudaError_t e;
        if (a.vtma) {
            const dim3 fg(static_cast<unsigned>(a.F),
                          static_cast<unsigned>((g.N + kFirThreads * kFirPts - 1) / (kFirThreads * kFirPts)));
            // hop == N: blocks shared by consecutive frames are read once;
            // the frame groups of a point range are consecutive CTAs, so the
            // blocks two groups share and the range's taps are read from
            // DRAM once (for N = 10^7 the taps alone are 160 MB)
            const dim3 fm(static_cast<unsigned>((a.F + kMfFrames - 1) / kMfFrames),
                          static_cast<unsigned>((g.N + kFirThreads * kMfPts - 1) / (kFirThreads * kMfPts)));
            const bool frames = a.sh_fixed >= 0 && a.hop == g.N;
            switch (frames ? a.T : -a.T) {
            case 2: gen_fir_frames_kernel<2><<<fm, kFirThreads, 0, st>>>(a); break;
            case 3: gen_fir_frames_kernel<3><<<fm, kFirThreads, 0, st>>>(a); break;
            case 4: gen_fir_frames_kernel<4><<<fm, kFirThreads, 0, st>>>(a); break;
            case 8: gen_fir_frames_kernel<8><<<fm, kFirThreads, 0, st>>>(a); break;
            case 1: case -1: gen_fir_kernel<1><<<fg, kFirThreads, 0, st>>>(a); break;
            case -2: gen_fir_kernel<2><<<fg, kFirThreads, 0, st>>>(a); break;
            case -3: gen_fir_kernel<3><<<fg, kFirThreads, 0, st>>>(a); break;
            case -4: gen_fir_kernel<4><<<fg, kFirThreads, 0, st>>>(a); break;
            case -8: gen_fir_kernel<8><<<fg, kFirThreads, 0, st>>>(a); break;
            default: gen_fir_kernel<0><<<fg, kFirThreads, 0, st>>>(a); break;
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        e = launch_gen<TH>(gen_pass_a_kernel<TH>, a.F * groups_a, g.N1 * ga, L.n_sms, st,
                           3 * kTwDigit * sizeof(float2) + 16, a, tmv);
        if (e != cudaSuccess) return e;
        e = launch_gen<TH>(gen_pass_b_kernel<TH>, a.F * groups_b, g.N2 * gb, L.n_sms, st, 16, a);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t gen_pfb_launch(const PfbLaunch& L, const GenPlan& g, cudaStream_t st) {
    if (L.F <= 0) return cudaSuccess;
    GenArgs a{};
    a.carry = reinterpret_cast<const uint32_t*>(L.carry);
    a.cl = L.cl;
    a.buf = reinterpret_cast<const uint32_t*>(L.buf);
    a.N = g.N;
    a.T = L.taps_kernel;
    a.hop = L.hop > 0 ? L.hop : g.N;
    a.gls = g.gls;
    a.a0 = L.a0;
    // frame starts a0 + k*N: one shift for every frame
    a.sh_fixed = a.hop == g.N ? static_cast<int>(((L.a0 % g.N) + g.N) % g.N) : -1;
    a.h = L.h;
    a.fa = g.fa;
    a.fb = g.fb;
    a.tw_a = g.d_tw;               // stage offsets of fa and fb index the one table
    a.tw_b = g.d_tw;
    a.tw3 = g.d_tw3;
    a.N1 = g.N1;
    a.N2 = g.N2;
    a.n2_magic = static_cast<uint32_t>(((uint64_t(1) << 32) + g.N2 - 1) / g.N2);
    a.gla = g.gla;
    a.glb = g.glb;
    a.z = g.d_z;
    a.bins = L.bins;
    a.n_tones = L.n_tones;
    a.gtone = g.d_gtone;
    a.goff = g.d_goff;
    // Z rows start on 16-byte boundaries when N and N2 are even (Z itself is
    // 256-byte aligned), and every copy is then a multiple of 16 bytes
    a.zbulk = (g.N % 2 == 0 && g.N2 % 2 == 0) ? 1 : 0;
    a.status = L.status;
    a.v = g.d_v;
    a.vtma = g.vtma;
    a.vbox_rows = g.vbox_rows;
    a.vboxes = g.vboxes;
    a.vsstride = g.vsstride;
    a.full = static_cast<float2*>(L.full);
    a.full_ld = L.full_ld;
    a.tones = static_cast<float2*>(L.tones);
    a.tones_ld = L.tones_ld;
    a.fo = L.frame_offset;
    auto fixed_id = [&](const GenFft& f, int gl2) {
        for (const FixedShape& c : kFixedShapes) {
            if (c.th != g.threads || c.gl2 != gl2 || c.n != f.n || c.nst != f.nst) continue;
            bool same = true;
            for (int s = 0; s < f.nst; ++s) same = same && c.radix[s] == f.radix[s];
            if (same) return c.id;
        }
        return 0;
    };
    a.fixa = g.N1 > 1 ? fixed_id(g.fa, g.gla) : 0;
    a.fixb = g.N1 > 1 ? fixed_id(g.fb, g.glb) : 0;
    return g.threads == 256 ? gen_run<256>(a, L, g, st) : gen_run<512>(a, L, g, st);
}

}  // namespace rfr
