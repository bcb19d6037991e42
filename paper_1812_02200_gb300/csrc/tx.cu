// tx.cu -- the transmit buffer (Sec. III: the GPU generates the transmission
// buffer as well as processing the received one): complex int16 samples of a
// multi-tone excitation built from the same NCO words the receiver
// demodulates,
//   s(m) = sum_t A_t exp(+i*2*pi*((w_t*m + p_t) mod 2^64) / 2^64),
// each component rounded half-to-even and clamped to int16.
//
// One thread computes 4 samples (m, m+256, m+512, m+768 of a 1024-sample
// tile); the tones stream through shared memory 256 at a time.  Per tone the
// thread forms the exact uint64 phase of its first sample and steps it by
// 256*w; the mixer is sincospif of the top 32 phase bits in FP32, summed in
// FP32 over chunks of 32 tones, the chunk sums added in FP64.
//
// Error of each component before rounding against the exact sum (see
// rfr_tx_error_bound):  e = sum_t A_t * (pi*(2^-25 + 2^-31)   angle: 32-bit
//                                         + 2^-23)              sincospif, 1 ulp
//                           + sum_t |fl(A_t) - A_t|             A_t rounded to FP32
//                           + sum_chunks k * 2^-24 * sum_chunk A  k FMA roundings
// plus FP64 rounding (< 2^-40 * sum A_t).  A component whose exact value lies
// farther than e from a rounding tie is therefore the exact rounding.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "../../include/rfr.h"
#include "trace.h"

namespace {

constexpr int kTxThreads = 256;
constexpr int kTxSpt = 4;                       // samples per thread per tile
constexpr int kTxTile = kTxThreads * kTxSpt;
constexpr int kTxChunk = 32;                    // tones per FP32 partial sum

__device__ __forceinline__ int16_t clamp_i16(double v) {
    return static_cast<int16_t>(fmin(fmax(v, -32768.0), 32767.0));
}

__global__ void __launch_bounds__(kTxThreads) tx_synth_kernel(const uint64_t* __restrict__ words,
                                                              const uint64_t* __restrict__ phases,
                                                              const float* __restrict__ amps, int nt,
                                                              int64_t m0, int64_t n, short2* __restrict__ out) {
    __shared__ uint64_t sw[kTxThreads], sp[kTxThreads];
    __shared__ float sa[kTxThreads];
    const int tid = threadIdx.x;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * kTxTile; base < n;
         base += static_cast<int64_t>(gridDim.x) * kTxTile) {
        const uint64_t mf = static_cast<uint64_t>(m0 + base + tid);    // first sample of this thread
        double acc_r[kTxSpt], acc_i[kTxSpt];
#pragma unroll
        for (int s = 0; s < kTxSpt; ++s) acc_r[s] = acc_i[s] = 0.0;
        for (int t0 = 0; t0 < nt; t0 += kTxThreads) {
            __syncthreads();
            if (t0 + tid < nt) {
                sw[tid] = __ldg(words + t0 + tid);
                sp[tid] = __ldg(phases + t0 + tid);
                sa[tid] = __ldg(amps + t0 + tid);
            }
            __syncthreads();
            const int cnt = min(kTxThreads, nt - t0);
            for (int c0 = 0; c0 < cnt; c0 += kTxChunk) {
                const int c1 = min(c0 + kTxChunk, cnt);
                float pr[kTxSpt], pi[kTxSpt];
#pragma unroll
                for (int s = 0; s < kTxSpt; ++s) pr[s] = pi[s] = 0.f;
                for (int t = c0; t < c1; ++t) {
                    const uint64_t w = sw[t];
                    const float a = sa[t];
                    uint64_t ph = w * mf + sp[t];
                    const uint64_t step = w * static_cast<uint64_t>(kTxThreads);
#pragma unroll
                    for (int s = 0; s < kTxSpt; ++s) {
                        float sn, cs;
                        sincospif(static_cast<float>(static_cast<int32_t>(ph >> 32)) * 0x1p-31f, &sn, &cs);
                        pr[s] = fmaf(a, cs, pr[s]);
                        pi[s] = fmaf(a, sn, pi[s]);
                        ph += step;
                    }
                }
#pragma unroll
                for (int s = 0; s < kTxSpt; ++s) {
                    acc_r[s] += static_cast<double>(pr[s]);
                    acc_i[s] += static_cast<double>(pi[s]);
                }
            }
        }
#pragma unroll
        for (int s = 0; s < kTxSpt; ++s) {
            const int64_t i = base + tid + static_cast<int64_t>(s) * kTxThreads;
            if (i < n) out[i] = make_short2(clamp_i16(rint(acc_r[s])), clamp_i16(rint(acc_i[s])));
        }
    }
}

}  // namespace

struct rfr_tx {
    int device = 0, n_sms = 0;
    int32_t n_tones = 0;
    uint64_t* d_words = nullptr;
    uint64_t* d_phases = nullptr;
    float* d_amps = nullptr;
    double error_bound = 0.0;
};

namespace {
void tx_free(rfr_tx* t) {
    if (!t) return;
    cudaFree(t->d_words);
    cudaFree(t->d_phases);
    cudaFree(t->d_amps);
    delete t;
}
}  // namespace

rfr_status rfr_tx_create(rfr_tx** out, const uint64_t* words, const uint64_t* phase_words, const double* amplitudes,
                         int32_t n_tones) {
    if (!out) return RFR_E_INVALID;
    *out = nullptr;
    if (n_tones < 1 || n_tones > 65536 || !words || !amplitudes) return RFR_E_INVALID;
    double sum = 0.0;
    for (int32_t t = 0; t < n_tones; ++t) {
        if (!(amplitudes[t] >= 0.0) || !std::isfinite(amplitudes[t])) return RFR_E_INVALID;
        sum += amplitudes[t];
    }
    if (sum > 1e6) return RFR_E_INVALID;
    rfr_tx* t = new (std::nothrow) rfr_tx();
    if (!t) return RFR_E_NOMEM;
    t->n_tones = n_tones;
    cudaGetDevice(&t->device);
    cudaDeviceGetAttribute(&t->n_sms, cudaDevAttrMultiProcessorCount, t->device);
    std::vector<uint64_t> ph(n_tones, 0);
    if (phase_words) std::copy(phase_words, phase_words + n_tones, ph.begin());
    std::vector<float> a(n_tones);
    double ea = 0.0;
    for (int32_t i = 0; i < n_tones; ++i) {
        a[i] = static_cast<float>(amplitudes[i]);
        ea += std::fabs(static_cast<double>(a[i]) - amplitudes[i]);
    }
    // per-term error, then k rounded FMA steps in each chunk of k tones (the
    // chunks the kernel forms: 32 at a time within each group of 256)
    double e = sum * (3.14159265358979 * (0x1p-25 + 0x1p-31) + 0x1p-23) + ea + sum * 0x1p-40;
    for (int32_t g0 = 0; g0 < n_tones; g0 += kTxThreads) {
        const int32_t g1 = std::min(n_tones, g0 + kTxThreads);
        for (int32_t c0 = g0; c0 < g1; c0 += kTxChunk) {
            const int32_t c1 = std::min(g1, c0 + kTxChunk);
            double sc = 0.0;
            for (int32_t i = c0; i < c1; ++i) sc += a[i];
            e += (c1 - c0) * 0x1p-24 * sc;
        }
    }
    t->error_bound = e;
    const size_t n8 = static_cast<size_t>(n_tones) * 8, n4 = static_cast<size_t>(n_tones) * 4;
    if (cudaMalloc(&t->d_words, n8) != cudaSuccess || cudaMalloc(&t->d_phases, n8) != cudaSuccess ||
        cudaMalloc(&t->d_amps, n4) != cudaSuccess) {
        tx_free(t);
        return RFR_E_NOMEM;
    }
    if (cudaMemcpy(t->d_words, words, n8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t->d_phases, ph.data(), n8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t->d_amps, a.data(), n4, cudaMemcpyHostToDevice) != cudaSuccess) {
        tx_free(t);
        return RFR_E_CUDA;
    }
    *out = t;
    return RFR_OK;
}

rfr_status rfr_tx_synthesize(rfr_tx* t, int64_t m0, int64_t n, int16_t* iq_out, void* stream) {
    rfr::TraceRange tr("rfr_tx_synthesize");
    if (!t || n < 0 || (n > 0 && !iq_out)) return RFR_E_INVALID;
    if (n == 0) return RFR_OK;
    const int64_t tiles = (n + kTxTile - 1) / kTxTile;
    const int64_t blocks = std::min<int64_t>(tiles, static_cast<int64_t>(t->n_sms) * 8);
    tx_synth_kernel<<<static_cast<unsigned>(blocks), kTxThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        t->d_words, t->d_phases, t->d_amps, t->n_tones, m0, n, reinterpret_cast<short2*>(iq_out));
    if (cudaGetLastError() != cudaSuccess) return RFR_E_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (rfr::debug_sync_allowed(st) && (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess))
        return RFR_E_CUDA;
    return RFR_OK;
}

double rfr_tx_error_bound(const rfr_tx* t) { return t ? t->error_bound : -1.0; }

void rfr_tx_destroy(rfr_tx* t) {
    if (t) cudaDeviceSynchronize();
    tx_free(t);
}
