// plain.cu -- the plain FP32 GPU forms used as the comparison baseline:
//   PFB:   an FP32 polyphase-FIR kernel writing the filtered frames, a batched
//          cuFFT C2C transform (the library route of Sec. III.A), and a gather
//          kernel for the tone bins;
//   demod: an FP32 CUDA-core kernel over the Toeplitz view of the stream with
//          FP32 modulated taps (mix + filter + decimate of Sec. III.B), or
//          cublasCgemm in pedantic FP32 (no TF32, no emulation) on the Toeplitz
//          matrix materialised in frame chunks (the library GEMM the paper
//          names for the same product).
// One-shot with zero history (frame k uses samples (k+1)*hop - W .. (k+1)*hop - 1).
#include <cublas_v2.h>
#include <cufft.h>

#include <algorithm>
#include <cstdint>

#include "dev_common.cuh"
#include "rfr_internal.h"

namespace rfr {

namespace {

__global__ void plain_fir_kernel(const uint32_t* __restrict__ x, int64_t n, int N, int T,
                                 const float* __restrict__ h, int64_t F, float2* __restrict__ v) {
    const int64_t total = F * N;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t k = i / N;
        const int p = static_cast<int>(i - k * N);
        const int64_t start = (k + 1) * N - static_cast<int64_t>(N) * T;
        float re = 0.f, im = 0.f;
        for (int t = 0; t < T; ++t) {
            const int64_t m = start + static_cast<int64_t>(t) * N + p;
            if (m < 0) continue;
            const float2 s = iq_to_f2(x[m]);
            const float c = h[t * N + p];
            re = fmaf(c, s.x, re);
            im = fmaf(c, s.y, im);
        }
        v[i] = make_float2(re, im);
    }
}

__global__ void plain_gather_kernel(const float2* __restrict__ y, int N, int64_t F,
                                    const int32_t* __restrict__ bins, int n_tones,
                                    float2* __restrict__ tones, int64_t ld) {
    const int64_t total = F * n_tones;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int s = static_cast<int>(i / F);
        const int64_t k = i - static_cast<int64_t>(s) * F;
        tones[s * ld + k] = y[k * N + bins[s]];
    }
}

__global__ void plain_copy_rows(const float2* __restrict__ y, int N, int64_t F, float2* __restrict__ out,
                                int64_t ld) {
    const int64_t total = F * N;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t k = i / N;
        out[k * ld + (i - k * N)] = y[i];
    }
}

unsigned grid_for(int64_t work) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 32)));
}

}  // namespace

cudaError_t plain_pfb(const int16_t* iq, int64_t n, int N, int T, const float* h, const int32_t* bins,
                      int n_tones, void* full, int64_t full_ld, void* tones, int64_t tones_ld,
                      void** scratch, size_t* scratch_bytes, void** fft_plan, int64_t* fft_batch,
                      cudaStream_t st) {
    const int64_t F = n / N;
    if (F <= 0) return cudaSuccess;
    const bool direct = full && full_ld == N;   // cuFFT can write straight into `full`
    const size_t need = static_cast<size_t>(F) * N * 8 * (direct ? 1 : 2);
    if (*scratch_bytes < need) {
        if (*scratch) cudaFree(*scratch);
        *scratch = nullptr;
        *scratch_bytes = 0;
        cudaError_t e = cudaMalloc(scratch, need);
        if (e != cudaSuccess) return e;
        *scratch_bytes = need;
    }
    float2* v = static_cast<float2*>(*scratch);
    float2* y = direct ? static_cast<float2*>(full) : v + F * N;
    if (*fft_batch != F * 33554432LL + N) {
        if (*fft_plan) {
            cufftDestroy(static_cast<cufftHandle>(reinterpret_cast<uintptr_t>(*fft_plan)));
            *fft_plan = nullptr;
        }
        cufftHandle ph;
        int dims[1] = {N};
        if (cufftPlanMany(&ph, 1, dims, nullptr, 1, N, nullptr, 1, N, CUFFT_C2C, static_cast<int>(F)) !=
            CUFFT_SUCCESS)
            return cudaErrorUnknown;
        *fft_plan = reinterpret_cast<void*>(static_cast<uintptr_t>(ph));
        *fft_batch = F * 33554432LL + N;
    }
    const cufftHandle ph = static_cast<cufftHandle>(reinterpret_cast<uintptr_t>(*fft_plan));
    cufftSetStream(ph, st);
    plain_fir_kernel<<<grid_for(F * N), 256, 0, st>>>(reinterpret_cast<const uint32_t*>(iq), n, N, T, h, F, v);
    if (cufftExecC2C(ph, reinterpret_cast<cufftComplex*>(v), reinterpret_cast<cufftComplex*>(y),
                     CUFFT_FORWARD) != CUFFT_SUCCESS)
        return cudaErrorUnknown;
    if (full && !direct)
        plain_copy_rows<<<grid_for(F * N), 256, 0, st>>>(y, N, F, static_cast<float2*>(full), full_ld);
    if (tones && n_tones > 0)
        plain_gather_kernel<<<grid_for(F * n_tones), 256, 0, st>>>(y, N, F, bins, n_tones,
                                                                     static_cast<float2*>(tones), tones_ld);
    return cudaGetLastError();
}

void plain_release(void* scratch, void* fft_plan, void* blas) {
    if (scratch) cudaFree(scratch);
    if (fft_plan) cufftDestroy(static_cast<cufftHandle>(reinterpret_cast<uintptr_t>(fft_plan)));
    if (blas) cublasDestroy(static_cast<cublasHandle_t>(blas));
}

}  // namespace rfr

// ------------------------------------------------------------- demod (FP32)
namespace rfr {
namespace {

__global__ void plain_taps_kernel(const float* __restrict__ h, const uint64_t* __restrict__ words,
                                  int n_tones, int L, float2* __restrict__ c) {
    const int64_t total = static_cast<int64_t>(n_tones) * L;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int t = static_cast<int>(i / L);
        const int n = static_cast<int>(i - static_cast<int64_t>(t) * L);
        const uint64_t ph = words[t] * static_cast<uint64_t>(n);
        double s, co;
        sincospi(static_cast<double>(static_cast<int64_t>(ph)) * 0x1p-63, &s, &co);
        c[i] = make_float2(static_cast<float>(h[n] * co), static_cast<float>(-h[n] * s));
    }
}

constexpr int PT = 64;     // frames and tones per block tile
constexpr int PK = 16;     // taps per k step

// out[t][k] = exp(-i*phi_t(b_k)) * sum_n x[b_k + n] * C_t[n], plain FP32 FMAs;
// each thread accumulates 4 frames x 4 tones.
__global__ void __launch_bounds__(256) plain_demod_kernel(const uint32_t* __restrict__ x, int64_t n_samples,
                                                          int L, int D, const float2* __restrict__ C,
                                                          const uint64_t* __restrict__ words, int n_tones,
                                                          int64_t F, float2* __restrict__ out, int64_t ld) {
    __shared__ float2 xs[PT][PK + 1];
    __shared__ float2 cs[PK][PT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t k0 = static_cast<int64_t>(blockIdx.x) * PT;
    const int t0 = blockIdx.y * PT;
    float2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int n0 = 0; n0 < L; n0 += PK) {
        for (int e = threadIdx.x; e < PT * PK; e += 256) {
            const int f = e / PK, j = e % PK;
            const int64_t k = k0 + f;
            const int64_t m = (k + 1) * D - L + n0 + j;
            float2 v = make_float2(0.f, 0.f);
            if (k < F && n0 + j < L && m >= 0 && m < n_samples) v = iq_to_f2(x[m]);
            xs[f][j] = v;
        }
        for (int e = threadIdx.x; e < PT * PK; e += 256) {
            const int j = e / PT, tt = e % PT;
            const int t = t0 + tt;
            cs[j][tt] = (t < n_tones && n0 + j < L) ? C[static_cast<int64_t>(t) * L + n0 + j] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < PK; ++j) {
            float2 xv[4], cv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) xv[a] = xs[ty + 16 * a][j];
#pragma unroll
            for (int b = 0; b < 4; ++b) cv[b] = cs[j][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc[a][b].x = fmaf(xv[a].x, cv[b].x, fmaf(-xv[a].y, cv[b].y, acc[a][b].x));
                    acc[a][b].y = fmaf(xv[a].x, cv[b].y, fmaf(xv[a].y, cv[b].x, acc[a][b].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t k = k0 + ty + 16 * a;
        if (k >= F) continue;
        const int64_t b_k = (k + 1) * D - L;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int t = t0 + tx + 16 * b;
            if (t >= n_tones) continue;
            const uint64_t ph = words[t] * static_cast<uint64_t>(b_k);
            float s, c;
            sincospif(static_cast<float>(static_cast<int32_t>(ph >> 32)) * 0x1p-31f, &s, &c);
            out[static_cast<int64_t>(t) * ld + k] = cmul(acc[a][b], make_float2(c, -s));
        }
    }
}

}  // namespace

cudaError_t plain_demod_taps(const float* h32, const uint64_t* words, int n_tones, int L, void* c32,
                             cudaStream_t st) {
    const int64_t total = static_cast<int64_t>(n_tones) * L;
    plain_taps_kernel<<<grid_for(total), 256, 0, st>>>(h32, words, n_tones, L, static_cast<float2*>(c32));
    return cudaGetLastError();
}

cudaError_t plain_demod(const int16_t* iq, int64_t n, int L, int D, const void* c32, const uint64_t* words,
                        int n_tones, void* tones, int64_t tones_ld, cudaStream_t st) {
    const int64_t F = n / D;
    if (F <= 0 || n_tones <= 0) return cudaSuccess;
    dim3 grid(static_cast<unsigned>((F + PT - 1) / PT), static_cast<unsigned>((n_tones + PT - 1) / PT));
    plain_demod_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const uint32_t*>(iq), n, L, D,
                                             static_cast<const float2*>(c32), words, n_tones, F,
                                             static_cast<float2*>(tones), tones_ld);
    return cudaGetLastError();
}

// ------------------------------------------------- demod (cublasCgemm, FP32)
namespace {

// X[r][n] = x[(k0 + r + 1) * D - L + n] as complex FP32, zero outside the buffer
// (frame k0 + r of the Toeplitz matrix; rows of L contiguous values).
__global__ void toeplitz_rows_kernel(const uint32_t* __restrict__ x, int64_t n_samples, int L, int D,
                                     int64_t k0, int64_t rows, float2* __restrict__ X) {
    const int64_t total = rows * L;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = i / L;
        const int64_t m = (k0 + r + 1) * D - L + (i - r * L);
        X[i] = (m >= 0 && m < n_samples) ? iq_to_f2(x[m]) : make_float2(0.f, 0.f);
    }
}

// out[t][k] *= exp(-i * phi_t(b_k)), b_k = (k + 1) * D - L, phase in uint64.
__global__ void rotate_rows_kernel(float2* __restrict__ out, int64_t ld, int64_t F, int L, int D,
                                   const uint64_t* __restrict__ words, int n_tones) {
    const int64_t total = F * n_tones;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int t = static_cast<int>(i / F);
        const int64_t k = i - static_cast<int64_t>(t) * F;
        const uint64_t ph = words[t] * static_cast<uint64_t>((k + 1) * D - L);
        float s, c;
        sincospif(static_cast<float>(static_cast<int32_t>(ph >> 32)) * 0x1p-31f, &s, &c);
        float2* o = out + static_cast<int64_t>(t) * ld + k;
        *o = cmul(*o, make_float2(c, -s));
    }
}

}  // namespace

cudaError_t plain_demod_cgemm(const int16_t* iq, int64_t n, int L, int D, const void* c32, const uint64_t* words,
                              int n_tones, void* tones, int64_t tones_ld, void** scratch, size_t* scratch_bytes,
                              void** blas, cudaStream_t st) {
    const int64_t F = n / D;
    if (F <= 0 || n_tones <= 0) return cudaSuccess;
    // frame chunk: the materialised rows take at most 512 MiB
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(F, (int64_t{512} << 20) / (int64_t{8} * L)));
    const size_t need = static_cast<size_t>(chunk) * L * 8;
    if (*scratch_bytes < need) {
        if (*scratch) cudaFree(*scratch);
        *scratch = nullptr;
        *scratch_bytes = 0;
        cudaError_t e = cudaMalloc(scratch, need);
        if (e != cudaSuccess) return e;
        *scratch_bytes = need;
    }
    if (!*blas) {
        cublasHandle_t h;
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
        if (cublasSetMathMode(h, CUBLAS_PEDANTIC_MATH) != CUBLAS_STATUS_SUCCESS) {
            cublasDestroy(h);
            return cudaErrorUnknown;
        }
        *blas = h;
    }
    cublasHandle_t h = static_cast<cublasHandle_t>(*blas);
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    float2* X = static_cast<float2*>(*scratch);
    float2* out = static_cast<float2*>(tones);
    const cuComplex one = make_cuComplex(1.f, 0.f), zero = make_cuComplex(0.f, 0.f);
    for (int64_t k0 = 0; k0 < F; k0 += chunk) {
        const int64_t rows = std::min(chunk, F - k0);
        toeplitz_rows_kernel<<<grid_for(rows * L), 256, 0, st>>>(reinterpret_cast<const uint32_t*>(iq), n, L, D,
                                                                  k0, rows, X);
        // column-major: Out (rows x tones, ld tones_ld) = X^T (rows x L) * C (L x tones); X and C
        // are row-major [rows][L] and [tone][L], i.e. column-major L x rows and L x tones.
        if (cublasCgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, static_cast<int>(rows), n_tones, L, &one,
                        reinterpret_cast<const cuComplex*>(X), L, static_cast<const cuComplex*>(c32), L, &zero,
                        reinterpret_cast<cuComplex*>(out + k0), static_cast<int>(tones_ld)) != CUBLAS_STATUS_SUCCESS)
            return cudaErrorUnknown;
    }
    rotate_rows_kernel<<<grid_for(F * n_tones), 256, 0, st>>>(out, tones_ld, F, L, D, words, n_tones);
    return cudaGetLastError();
}

}  // namespace rfr
