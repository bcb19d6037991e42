// fft_dev.cuh -- in-CTA FP32 FFT of one PFB frame (the "batched FFT" step of
// Sec. III.A, done per frame in registers and shared memory).
//
// Layout: a frame of N = 2^LOG2N points is handled by NT = N/16 threads, 16
// points per thread.  The transform is a Stockham autosort FFT: radix-16
// passes first, then one radix-2/4/8 pass if LOG2N is not a multiple of 4.
// Pass with radix R and span Ns (product of the radices already done): the
// butterfly j reads x[j + r*N/R] (r < R), multiplies by W_{R*Ns}^{r*k} with
// k = j mod Ns, does a length-R DFT and writes y[(j/Ns)*R*Ns + k + r*Ns].
// Forward sign exp(-2*pi*i/N), natural order in and out, no scaling.
//
// Between passes the frame goes through a shared-memory buffer whose index is
// padded by one element every 16 (pad(i) = i + i/16), which keeps every
// access pattern of the passes free of bank conflicts.
//
// Twiddles are FP32 values of FP64-evaluated exp(-2*pi*i*m/L), precomputed
// on the host per pass as table[(r-1)*Ns + k] (see pfb_twiddle_count).
#pragma once
#include "dev_common.cuh"

namespace rfr {

__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }

__device__ __forceinline__ void dft2(float2& a, float2& b) {
    const float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
    const float2 t0 = cadd(x0, x2), t1 = csub(x0, x2);
    const float2 t2 = cadd(x1, x3), t3 = cmul_mi(csub(x1, x3));
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

constexpr float kC8 = 0.92387953251128674f;   // cos(pi/8)
constexpr float kS8 = 0.38268343236508977f;   // sin(pi/8)
constexpr float kR2 = 0.70710678118654752f;   // sqrt(1/2)

// a * exp(-i*pi/4)
__device__ __forceinline__ float2 cmul_w8(float2 a) {
    return make_float2((a.x + a.y) * kR2, (a.y - a.x) * kR2);
}
// a * exp(-3i*pi/4)
__device__ __forceinline__ float2 cmul_w8_3(float2 a) {
    return make_float2((a.y - a.x) * kR2, -(a.x + a.y) * kR2);
}

// x[0..7] -> DFT8, natural order.
__device__ __forceinline__ void dft8(float2* x) {
    float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    float2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dft4(e0, e1, e2, e3);
    dft4(o0, o1, o2, o3);
    o1 = cmul_w8(o1);
    o2 = cmul_mi(o2);
    o3 = cmul_w8_3(o3);
    x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
    x[1] = cadd(e1, o1); x[5] = csub(e1, o1);
    x[2] = cadd(e2, o2); x[6] = csub(e2, o2);
    x[3] = cadd(e3, o3); x[7] = csub(e3, o3);
}

// x[0..15] -> DFT16, natural order (4 x 4 decomposition, n = 4*n1 + n2,
// X[k1 + 4*k2]).
__device__ __forceinline__ void dft16(float2* x) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
    // x[4*k1 + n2] *= W16^(n2*k1)
    const float2 w1 = make_float2(kC8, -kS8), w3 = make_float2(kS8, -kC8);
    const float2 w9 = make_float2(-kC8, kS8);
    x[5] = cmul(x[5], w1);
    x[9] = cmul_w8(x[9]);
    x[13] = cmul(x[13], w3);
    x[6] = cmul_w8(x[6]);
    x[10] = cmul_mi(x[10]);
    x[14] = cmul_w8_3(x[14]);
    x[7] = cmul(x[7], w3);
    x[11] = cmul_w8_3(x[11]);
    x[15] = cmul(x[15], w9);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
    // position 4*k1 + k2 holds X[k1 + 4*k2]: transpose 4x4
    float2 y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = x[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = y[i];
}

template <int R>
__device__ __forceinline__ void dft_small(float2* x) {
    if constexpr (R == 2) dft2(x[0], x[1]);
    else if constexpr (R == 4) dft4(x[0], x[1], x[2], x[3]);
    else if constexpr (R == 8) dft8(x);
    else dft16(x);
}

// Number of FP32 complex twiddles the passes of an N-point frame use.
__host__ __device__ constexpr int pfb_twiddle_count(int log2n) {
    int cnt = 0, ns = 16;
    const int p16 = log2n / 4, rf = 1 << (log2n % 4);
    for (int s = 1; s < p16; ++s, ns *= 16) cnt += 15 * ns;
    if (rf > 1) cnt += (rf - 1) * ((1 << log2n) / rf);
    return cnt;
}

// Twiddle loader: shared-memory table or read-only global table.
template <bool SMEM>
__device__ __forceinline__ float2 tw_load(const float2* t, int i) {
    if constexpr (SMEM) return t[i];
    else return __ldg(t + i);
}

// The FFT of one frame.  On entry v[r] = x[tf + r*NT] (the thread's 16
// polyphase outputs).  On exit v holds y at the indices given by
// fft_out_index(), and nothing of the spectrum is in `buf` (the caller stores
// it there if it needs it).  All CTA threads must call this together (it
// contains __syncthreads); threads of masked frames still call it.
template <int LOG2N, bool TW_SMEM>
__device__ __forceinline__ void fft_frame(float2 (&v)[16], float2* buf, int tf,
                                          const float2* tw) {
    constexpr int N = 1 << LOG2N;
    constexpr int NT = N / 16;
    constexpr int P16 = LOG2N / 4;
    constexpr int RF = 1 << (LOG2N % 4);
    static_assert(LOG2N >= 4, "N >= 16");

    dft16(v);  // pass 0, span 1
    if constexpr (P16 > 1 || RF > 1) {   // N = 16: one pass only
        // write y[16*tf + r]
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[fpad(16 * tf + r)] = v[r];
        int tw_off = 0;
#pragma unroll
        for (int s = 1; s < P16; ++s) {
            const int ns = 1 << (4 * s);
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = buf[fpad(tf + r * NT)];
            const int k = tf & (ns - 1);
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw_load<TW_SMEM>(tw, tw_off + (r - 1) * ns + k));
            tw_off += 15 * ns;
            dft16(v);
            const bool last = (s == P16 - 1) && (RF == 1);
            if (!last) {
                __syncthreads();
                const int base = (tf / ns) * 16 * ns + k;
#pragma unroll
                for (int r = 0; r < 16; ++r) buf[fpad(base + r * ns)] = v[r];
            }
        }
        if constexpr (RF > 1) {
            constexpr int NB = 16 / RF;      // butterflies per thread
            constexpr int SPAN = N / RF;     // Ns of the final pass
            __syncthreads();
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int j = tf + q * NT;
#pragma unroll
                for (int r = 0; r < RF; ++r) v[q * RF + r] = buf[fpad(j + r * SPAN)];
#pragma unroll
                for (int r = 1; r < RF; ++r)
                    v[q * RF + r] = cmul(v[q * RF + r], tw_load<TW_SMEM>(tw, tw_off + (r - 1) * SPAN + j));
                dft_small<RF>(v + q * RF);
            }
        }
    }
}

// Output index (bin) held in v[i] after fft_frame.
template <int LOG2N>
__device__ __forceinline__ int fft_out_index(int tf, int i) {
    constexpr int N = 1 << LOG2N;
    constexpr int NT = N / 16;
    constexpr int RF = 1 << (LOG2N % 4);
    if constexpr (RF == 1) {
        return tf + i * NT;
    } else {
        const int q = i / RF, r = i % RF;
        return tf + q * NT + r * (N / RF);
    }
}

}  // namespace rfr
