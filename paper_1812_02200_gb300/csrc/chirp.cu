// chirp.cu -- the chirped readout (Sec. III.C, Eq. 1).
//
// Eq. 1, phi_t = 2*pi*(f0*t + k*t^2), in sample units t = m/fs becomes the
// exact uint64 phase  p(m) = s*m + r*m^2 (mod 2^64)  in units of 2*pi/2^64,
// s = f0/fs*2^64 (start word), r = k/fs^2*2^64 (rate word).
//
// chirp_synth_kernel: the transmit buffer generated on the GPU in real time
// (instead of a stored table): round-half-even of A*cos, A*sin of the phase,
// as complex int16.  The sine and cosine are computed in FP32 (the paper's
// "32 bit precision"); a component whose FP32 value lies within twice its
// error bound of a rounding tie is recomputed in FP64, so every int16 is the
// FP64 decision.
//
// chirp_demod_kernel: demodulation of the Rx stream against chirps ("using
// the algorithm outlined in section III.B"): for chirp c and frame k,
//   out[c][k] = sum_{n<L} h[n] x[b_k+n] exp(-i*2*pi*p_c(b_k+n)/2^64),
// the mix fused into the filter (the mixer depends on the frame through the
// quadratic term, so there is no fixed modulated-tap matrix to multiply).
// One CTA per frame, all chirps: each thread mixes and filters L/256 taps per
// chirp in FP32; the partial sums are reduced in FP32 within a warp and in FP64
// across the warps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "dev_common.cuh"
#include "rfr_internal.h"

namespace rfr {

namespace {

__device__ __forceinline__ uint64_t chirp_phase(uint64_t s, uint64_t r, int64_t m) {
    const uint64_t um = static_cast<uint64_t>(m);
    return s * um + r * (um * um);
}

// ---------------------------------------------------------------- synthesis
//
// A sample is A*exp(i*2*pi*p/2^64).  The phase is reduced exactly to the
// nearest quarter turn q and an offset x in [-1/4, 1/4] (angle / pi), taken
// from the top 32 phase bits and rounded to 24 significant bits (error
// <= 2^-27 + 2^-31).  Error of the FP32 value v = fl(fl(A) * sincospif(x))
// against A*sin (or cos) of the exact angle, |v - v_exact| <= e with
//   e = A*(pi*(2^-27 + 2^-31) + 2^-24 + 2^-24) + |fl(A) - A|
// (argument rounding, 1 ulp of sincospif for results below 1 in magnitude,
// product rounding).  When |v - rint(v)| <= 1/2 - 2e, rint(v) is the rounding
// of the exact value; every other component goes to a per-tile queue in
// shared memory and is recomputed in FP64 (sincos_phase_f64) by the whole
// CTA, so the FP64 pipe only ever runs full warps (its throughput is counted
// per warp instruction, active lanes or not).
constexpr int kSynThreads = 256;
constexpr int kSynTile = 2048;          // samples per tile (8 per thread)

__device__ __forceinline__ int16_t clamp16(float v) {
    return static_cast<int16_t>(fminf(fmaxf(v, -32768.f), 32767.f));
}

// FP64 sine and cosine of the exact phase for the near-tie recompute, from
// the angle-addition formula: the phase is reduced in integer arithmetic to a
// quarter turn q, an offset i/1024 of a half turn (|i| <= 256, table of FP64
// sin and cos of pi*i/1024) and a remainder delta, |delta| <= pi/2048, whose
// sine and cosine come from their Taylor series (terms to delta^7 and
// delta^8: truncation below 1e-25).
struct SinCos1024 {
    double s[513], c[513];
};
__device__ SinCos1024 g_sc1024;

__device__ __forceinline__ void sincos_phase_f64(uint64_t p, const double2* __restrict__ tab, double* sn,
                                                 double* cs) {
    const uint32_t q = static_cast<uint32_t>((p + (1ull << 61)) >> 62);
    const int64_t f = static_cast<int64_t>(p - (static_cast<uint64_t>(q) << 62));     // x = f / 2^63
    const int64_t i = (f + (int64_t(1) << 52)) >> 53;                                 // nearest i/1024
    const int64_t r = f - i * (int64_t(1) << 53);                                     // |r| <= 2^52
    const double d = static_cast<double>(r) * 3.4061215800865545e-19;                 // pi * 2^-63
    const double d2 = d * d;
    const double sd = d * (1.0 + d2 * (-1.0 / 6 + d2 * (1.0 / 120 + d2 * (-1.0 / 5040))));
    const double cd = 1.0 + d2 * (-0.5 + d2 * (1.0 / 24 + d2 * (-1.0 / 720 + d2 * (1.0 / 40320))));
    const double2 t = tab[i + 256];                                                   // (sin, cos)
    double sx = fma(t.x, cd, t.y * sd), cx = fma(t.y, cd, -(t.x * sd));
    if (q & 1) {
        const double u = sx;
        sx = cx;
        cx = -u;
    }
    if (q & 2) {
        sx = -sx;
        cx = -cx;
    }
    *sn = sx;
    *cs = cx;
}

__global__ void __launch_bounds__(kSynThreads) chirp_synth_kernel(uint64_t s, uint64_t r, float ampf,
                                                                  double amp, float tie_lo, int64_t m0,
                                                                  int64_t n, short2* __restrict__ out) {
    __shared__ __align__(16) short2 tile[kSynTile];
    __shared__ uint16_t fix[2 * kSynTile];
    __shared__ int nfix;
    __shared__ double2 tab[513];
    const int tid = threadIdx.x;
    for (int i = tid; i < 513; i += kSynThreads) tab[i] = make_double2(g_sc1024.s[i], g_sc1024.c[i]);
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * kSynTile; base < n;
         base += static_cast<int64_t>(gridDim.x) * kSynTile) {
        if (tid == 0) nfix = 0;
        __syncthreads();
        const int cnt = static_cast<int>(n - base < kSynTile ? n - base : kSynTile);
        // p(m + 256) = p(m) + d(m), d(m + 256) = d(m) + 2*256^2*r  (all mod 2^64)
        const uint64_t m = static_cast<uint64_t>(m0 + base + tid);
        uint64_t p = chirp_phase(s, r, static_cast<int64_t>(m));
        uint64_t d = s * 256ull + r * (512ull * m + 65536ull);
        const uint64_t dd = r * 131072ull;
        for (int i = tid; i < cnt; i += kSynThreads) {
            // quarter turn q and offset from the top 32 phase bits:
            // x = fi * 2^-31 in [-1/4, 1/4] (angle / pi)
            const uint32_t hi = static_cast<uint32_t>(p >> 32);
            const uint32_t q = ((hi + (1u << 29)) >> 30) & 3u;
            const int32_t fi = static_cast<int32_t>(hi - (q << 30));
            float sx, cx;
            sincospif(static_cast<float>(fi) * 0x1p-31f, &sx, &cx);
            float c = cx, sn = sx;                 // rotate by q quarter turns
            if (q & 1) {
                c = -sx;
                sn = cx;
            }
            if (q & 2) {
                c = -c;
                sn = -sn;
            }
            const float vc = ampf * c, vs = ampf * sn;
            const float rc = rintf(vc), rs = rintf(vs);
            if (fabsf(vc - rc) > tie_lo) fix[atomicAdd(&nfix, 1)] = static_cast<uint16_t>(i << 1);
            if (fabsf(vs - rs) > tie_lo) fix[atomicAdd(&nfix, 1)] = static_cast<uint16_t>((i << 1) | 1);
            tile[i] = make_short2(clamp16(rc), clamp16(rs));
            p += d;
            d += dd;
        }
        __syncthreads();
        const int nf = nfix;
        int16_t* comp = reinterpret_cast<int16_t*>(tile);
        for (int j = tid; j < nf; j += kSynThreads) {
            const int e = fix[j];
            double sd, cd;
            sincos_phase_f64(chirp_phase(s, r, m0 + base + (e >> 1)), tab, &sd, &cd);
            comp[e] = clamp16(static_cast<float>(rint(amp * ((e & 1) ? sd : cd))));
        }
        __syncthreads();
        short2* dst = out + base;
        if (cnt == kSynTile && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
            const uint4* src4 = reinterpret_cast<const uint4*>(tile);
            uint4* dst4 = reinterpret_cast<uint4*>(dst);
            for (int i = tid; i < kSynTile / 4; i += kSynThreads) dst4[i] = src4[i];
        } else {
            for (int i = tid; i < cnt; i += kSynThreads) dst[i] = tile[i];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------- demodulation
//
// One CTA per frame (grid-stride): the frame's L samples are converted to FP32
// once into shared memory and reused by every chirp.  For chirp c a thread
// walks its taps n = tid, tid + 256, ... with the exact phase recurrence
// p(m + 256) = p(m) + d, d += 2*256^2*r; the mixer is sincospif of the top 32
// bits in FP32 and the products are summed in FP32 per thread and across the
// warp (shuffles); the 8 warp sums are added in FP64 (through shared memory,
// a group of 32 chirps at a time).
constexpr int kChirpThreads = 256;
constexpr int kChirpGroup = 32;

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
    extern __shared__ float2 xs[];                      // [L]
    __shared__ double2 red[kChirpGroup][kChirpThreads / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int64_t k = blockIdx.x; k < a.F; k += gridDim.x) {
        __syncthreads();                                // previous frame's readers are done
        for (int n = tid; n < a.L; n += kChirpThreads) {
            const int64_t vi = k * a.D + n;             // index in [carry | buffer]
            xs[n] = iq_to_f2(vi < a.cl ? __ldg(a.carry + vi) : __ldg(a.buf + (vi - a.cl)));
        }
        __syncthreads();
        const uint64_t m = static_cast<uint64_t>(a.a0 + k * a.D + tid);
        for (int c0 = 0; c0 < a.n_chirps; c0 += kChirpGroup) {
            const int cn = a.n_chirps - c0 < kChirpGroup ? a.n_chirps - c0 : kChirpGroup;
            for (int cc = 0; cc < cn; ++cc) {
                const uint64_t s = __ldg(a.s + c0 + cc), r = __ldg(a.r + c0 + cc);
                uint64_t p = chirp_phase(s, r, static_cast<int64_t>(m));
                uint64_t d = s * 256ull + r * (512ull * m + 65536ull);
                const uint64_t dd = r * 131072ull;
                float ar = 0.f, ai = 0.f;
                for (int n = tid; n < a.L; n += kChirpThreads) {
                    const float2 x = xs[n];
                    float sn, cs;
                    sincospif(static_cast<float>(static_cast<int32_t>(p >> 32)) * 0x1p-31f, &sn, &cs);
                    // x * exp(-i*theta) = (x.re*cos + x.im*sin, x.im*cos - x.re*sin)
                    const float mr = fmaf(x.x, cs, x.y * sn), mi = fmaf(x.y, cs, -x.x * sn);
                    const float hn = __ldg(a.h + n);
                    ar = fmaf(hn, mr, ar);
                    ai = fmaf(hn, mi, ai);
                    p += d;
                    d += dd;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    ar += __shfl_xor_sync(0xffffffffu, ar, o);
                    ai += __shfl_xor_sync(0xffffffffu, ai, o);
                }
                if (lane == 0) red[cc][warp] = make_double2(ar, ai);
            }
            __syncthreads();
            if (tid < cn) {
                double tr = 0.0, ti = 0.0;
                for (int w = 0; w < kChirpThreads / 32; ++w) {
                    tr += red[tid][w].x;
                    ti += red[tid][w].y;
                }
                a.out[static_cast<int64_t>(c0 + tid) * a.ld + a.fo + k] =
                    make_float2(static_cast<float>(tr), static_cast<float>(ti));
            }
            __syncthreads();
        }
    }
}

}  // namespace

namespace {
// The FP64 sine/cosine table of the near-tie recompute, uploaded once per
// device (the first synthesis on a device; call it outside stream capture).
std::mutex g_sc_mu;
bool g_sc_done[64] = {};

cudaError_t ensure_sincos_table() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_sc_mu);
    if (g_sc_done[dev]) return cudaSuccess;
    SinCos1024 t;
    for (int i = -256; i <= 256; ++i) {
        t.s[i + 256] = std::sin(3.14159265358979323846 * i / 1024.0);
        t.c[i + 256] = std::cos(3.14159265358979323846 * i / 1024.0);
    }
    e = cudaMemcpyToSymbol(g_sc1024, &t, sizeof(t));
    if (e == cudaSuccess) g_sc_done[dev] = true;
    return e;
}
}  // namespace

cudaError_t chirp_synth(uint64_t s, uint64_t r, double amp, int64_t m0, int64_t n, void* out,
                        cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const float ampf = static_cast<float>(amp);
    // argument rounding, 1 ulp of sincospif (results below 1 in magnitude:
    // 2^-24), product rounding, amplitude rounding
    const double e = amp * (3.14159265358979 * (0x1p-27 + 0x1p-31) + 0x1p-24 + 0x1p-24) +
                     std::fabs(static_cast<double>(ampf) - amp);
    cudaError_t ce = ensure_sincos_table();
    if (ce != cudaSuccess) return ce;
    const float tie_lo = static_cast<float>(0.5 - 2.0 * e);
    const int64_t tiles = (n + kSynTile - 1) / kSynTile;
    const int64_t blocks = std::min<int64_t>(tiles, 152 * 8);
    chirp_synth_kernel<<<static_cast<unsigned>(blocks), kSynThreads, 0, st>>>(
        s, r, ampf, amp, tie_lo, m0, n, static_cast<short2*>(out));
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
    const size_t smem = static_cast<size_t>(L.L) * sizeof(float2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(chirp_demod_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    const int per_sm = std::max(1, std::min(8, static_cast<int>((220u * 1024u) / (smem + 5u * 1024u))));
    const int64_t blocks = std::min<int64_t>(L.F, static_cast<int64_t>(L.n_sms) * per_sm);
    chirp_demod_kernel<<<static_cast<unsigned>(blocks), kChirpThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace rfr
