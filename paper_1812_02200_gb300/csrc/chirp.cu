// chirp.cu -- the chirped readout (Sec. III.C, Eq. 1).
//
// Eq. 1, phi_t = 2*pi*(f0*t + k*t^2), in sample units t = m/fs becomes the
// exact uint64 phase  p(m) = s*m + r*m^2 (mod 2^64)  in units of 2*pi/2^64,
// s = f0/fs*2^64 (start word), r = k/fs^2*2^64 (rate word).
//
// chirp_synth_kernel: the transmit buffer generated on the GPU in real time
// (instead of a stored table): round-half-even of A*cos, A*sin of the phase,
// as complex int16.  The sine and cosine are computed in FP32 (the paper's
// "32 bit precision"); a sample whose FP32 value lies within 0.02 of a
// rounding tie is recomputed in FP64, so every int16 is the FP64 decision.
//
// chirp_demod_kernel: demodulation of the Rx stream against chirps ("using
// the algorithm outlined in section III.B"): for chirp c and frame k,
//   out[c][k] = sum_{n<L} h[n] x[b_k+n] exp(-i*2*pi*p_c(b_k+n)/2^64),
// the mix fused into the filter (the mixer depends on the frame through the
// quadratic term, so there is no fixed modulated-tap matrix to multiply).
// One CTA per (chirp, frame): each thread mixes and filters L/256 taps in
// FP32; the partial sums are reduced in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "dev_common.cuh"
#include "rfr_internal.h"

namespace rfr {

namespace {

__device__ __forceinline__ uint64_t chirp_phase(uint64_t s, uint64_t r, int64_t m) {
    const uint64_t um = static_cast<uint64_t>(m);
    return s * um + r * (um * um);
}

// One component: round-half-even of v32 unless it is near a tie, in which
// case the FP64 value decides; clamped to int16.
__device__ __forceinline__ int16_t round_component(float v32, double amp, double unit, bool is_sin) {
    const float r32 = rintf(v32);
    float v = r32;
    if (fabsf(v32 - r32) > 0.48f) {
        double s, c;
        sincospi(unit, &s, &c);
        v = static_cast<float>(rint(amp * (is_sin ? s : c)));
    }
    v = fminf(fmaxf(v, -32768.f), 32767.f);
    return static_cast<int16_t>(v);
}

__global__ void chirp_synth_kernel(uint64_t s, uint64_t r, double amp, int64_t m0, int64_t n,
                                   short2* __restrict__ out) {
    const float ampf = static_cast<float>(amp);
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint64_t p = chirp_phase(s, r, m0 + i);
        // angle / pi in [-1, 1): FP32 from the top 32 bits, FP64 from all 64
        const float x32 = static_cast<float>(static_cast<int32_t>(p >> 32)) * 0x1p-31f;
        float sn, cs;
        sincospif(x32, &sn, &cs);
        const double x64 = static_cast<double>(static_cast<int64_t>(p)) * 0x1p-63;
        out[i] = make_short2(round_component(ampf * cs, amp, x64, false),
                             round_component(ampf * sn, amp, x64, true));
    }
}

constexpr int kChirpThreads = 256;

struct ChirpArgs {
    const uint32_t* carry;
    int64_t cl;
    const uint32_t* buf;
    int64_t F;
    int64_t a0;             // absolute sample index of v[0]
    int L, D;
    const float* h;
    const uint64_t* s;
    const uint64_t* r;
    int n_chirps;
    float2* out;
    int64_t ld, fo;
};

__global__ void __launch_bounds__(kChirpThreads) chirp_demod_kernel(const ChirpArgs a) {
    __shared__ double red[2][kChirpThreads / 32];
    const int64_t items = a.F * a.n_chirps;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int c = static_cast<int>(it / a.F);
        const int64_t k = it - static_cast<int64_t>(c) * a.F;
        const uint64_t s = __ldg(a.s + c), r = __ldg(a.r + c);
        float ar = 0.f, ai = 0.f;
        for (int n = threadIdx.x; n < a.L; n += kChirpThreads) {
            const int64_t vi = k * a.D + n;                          // index in [carry | buffer]
            const uint32_t w = vi < a.cl ? __ldg(a.carry + vi) : __ldg(a.buf + (vi - a.cl));
            const float2 x = iq_to_f2(w);
            const uint64_t p = chirp_phase(s, r, a.a0 + vi);
            float sn, cs;
            sincospif(static_cast<float>(static_cast<int32_t>(p >> 32)) * 0x1p-31f, &sn, &cs);
            // x * exp(-i*theta) = (x.re*cos + x.im*sin, x.im*cos - x.re*sin)
            const float mr = fmaf(x.x, cs, x.y * sn), mi = fmaf(x.y, cs, -x.x * sn);
            const float hn = __ldg(a.h + n);
            ar = fmaf(hn, mr, ar);
            ai = fmaf(hn, mi, ai);
        }
        double dr = ar, di = ai;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dr += __shfl_xor_sync(0xffffffffu, dr, o);
            di += __shfl_xor_sync(0xffffffffu, di, o);
        }
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) {
            red[0][warp] = dr;
            red[1][warp] = di;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double tr = 0.0, ti = 0.0;
            for (int w8 = 0; w8 < kChirpThreads / 32; ++w8) {
                tr += red[0][w8];
                ti += red[1][w8];
            }
            a.out[static_cast<int64_t>(c) * a.ld + a.fo + k] = make_float2(static_cast<float>(tr), static_cast<float>(ti));
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t chirp_synth(uint64_t s, uint64_t r, double amp, int64_t m0, int64_t n, void* out,
                        cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    chirp_synth_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(s, r, amp, m0, n,
                                                                       static_cast<short2*>(out));
    return cudaGetLastError();
}

cudaError_t chirp_demod_launch(const ChirpLaunch& L, cudaStream_t st) {
    if (L.F <= 0 || L.n_chirps <= 0) return cudaSuccess;
    ChirpArgs a{};
    a.carry = reinterpret_cast<const uint32_t*>(L.carry);
    a.cl = L.cl;
    a.buf = reinterpret_cast<const uint32_t*>(L.buf);
    a.F = L.F;
    a.a0 = L.a0;
    a.L = L.L;
    a.D = L.D;
    a.h = L.h32;
    a.s = L.start_words;
    a.r = L.rate_words;
    a.n_chirps = L.n_chirps;
    a.out = static_cast<float2*>(L.tones);
    a.ld = L.tones_ld;
    a.fo = L.frame_offset;
    const int64_t items = L.F * L.n_chirps;
    const int64_t blocks = std::min<int64_t>(items, static_cast<int64_t>(L.n_sms) * 8);
    chirp_demod_kernel<<<static_cast<unsigned>(blocks), kChirpThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace rfr
