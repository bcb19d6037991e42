// pfb_kernels.cu -- the polyphase filter bank of Sec. III.A of
// arXiv:1812.02200 for power-of-two N: int16 IQ -> FP32 polyphase FIR ->
// N-point FFT -> full spectrum and/or tone-bin gather.
//
// Stream view.  A push sees the virtual stream v = [carry | buffer]: `carry`
// (plan-owned, device) holds the last W - N + r samples of the stream (zero
// history at the start, r = partial-frame residue) and `buffer` the caller's
// new samples.  Frame j of the push (0 <= j < F) uses v-blocks j .. j+T-1,
// where v-block b is v[b*N, (b+1)*N):
//     v_j[p] = sum_{t<T} h[t*N + p] * v[(j+t)*N + p]
//     y_j[c] = sum_p v_j[p] exp(-2*pi*i*c*p/N)
// which is frame (F0 + j) of the stream, F0 the frames before this push.
//
// Kernels:
//  TMEM   (N = 4096, T <= 8, 16-byte aligned pushes): the FP32 delay line in
//         tensor memory, int16 blocks by 1-D TMA, spectrum rows by TMA bulk
//         stores and tone groups by 2-D TMA tensor stores (see below); the
//         symmetric-tap form (exactly symmetric taps, the plan default) pairs
//         mirrored rows per lane pair and also runs the phase passes of
//         oversampled plans; a seeded form continues FIR sums from pre-sum
//         rows (N = 4096 with 9..16 taps: first-half pass + taps 8..15).
//  RING   (N <= 4096, T <= 8 after padding): each CTA owns a contiguous run
//         of "super-blocks" (4096 samples = G = 4096/N frames' worth of new
//         samples).  A ring of super-blocks in shared memory is filled by
//         1-D TMA bulk copies (cp.async.bulk + mbarrier complete_tx), P
//         super-blocks ahead; each sample is read from HBM once.  The FIR
//         taps of the thread's 16 branches live in registers.
//  CLUSTER (N = 8192, 16384, T <= 8; a plan choice): N/4096 CTAs per frame
//         sharing the FFT through distributed shared memory.
//  DIRECT (any other N <= 16384, T <= 16): the in-CTA FFT per frame, its FIR
//         either a separate DRAM-streaming pre-sum pass (fir_pre_kernel; N =
//         8192, 16384 with T > 4, N = 256 .. 2048 with T > 8) or read from
//         global memory inside the kernel (L2 serves the T-fold reuse).
// RING and DIRECT run the in-CTA FFT of fft_dev.cuh (TMEM the same passes
// written out for N = 4096); all write
//   full[(frame_offset + j) * full_ld + c]      (natural bin order)
//   tones[s * tones_ld + frame_offset + j] = y_j[bin[s]].
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "dev_common.cuh"
#include "fft_dev.cuh"
#include "rfr_internal.h"
#include "umma.cuh"

namespace rfr {

constexpr int kSB = 4096;          // samples per super-block (16 KiB of IQ)
constexpr int kRingThreads = 256;

struct PfbArgs {
    const uint32_t* carry;   // packed IQ words
    int64_t cl;              // carry length (samples)
    const uint32_t* buf;
    int64_t n;               // buffer length (samples)
    int64_t F;               // frames to produce
    const float* h;          // taps [T*N] (kernel T)
    const float2* tw;        // FFT twiddles
    int tw_count;
    int T;                   // kernel taps (DIRECT variant)
    const int32_t* bins;
    int n_tones;
    float2* full;
    int64_t full_ld;
    float2* tones;
    int64_t tones_ld;
    int64_t frame_offset;
    int use_tma;
    int tones_tma;           // TMEM variant: whole tone groups leave by 2-D TMA stores
    int nb_smem;             // TMEM variant: tones staged in smem (0 or n_tones)
    int full_bulk;           // TMEM variant: full rows written by one TMA bulk store each
    int* status;
    int tone_cs;             // symmetric-tap kernel: tone columns of consecutive frames this far apart
    int rot;                 // symmetric-tap kernel: bin c multiplied by (-i)^((c * rot) mod 4)
    const float2* pre;       // TMEM kernel <T, true>: [F][4096] FIR partial sums the frames' FIR starts from
    int64_t q_lo, q_hi;      // iteration range
    int64_t iters_per_cta;
    int ring_sb;             // RING: super-blocks in the ring
};

__host__ __device__ __forceinline__ int64_t min_i64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max_i64(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ uint32_t vload(const PfbArgs& a, int64_t idx) {
    return idx < a.cl ? __ldg(a.carry + idx) : __ldg(a.buf + (idx - a.cl));
}

// Copies super-block q (its needed part) of v into ring slot `dst`.
// TMA path: one elected thread, completion on `bar`.
__device__ __forceinline__ void issue_sb_tma(const PfbArgs& a, int64_t q, int64_t need,
                                             uint32_t* dst, uint64_t* bar) {
    const int64_t lo = q * kSB;
    const int64_t hi = min(lo + kSB, need);
    const uint32_t bytes = static_cast<uint32_t>(hi - lo) * 4u;
    mbar_arrive_expect_tx(bar, bytes);
    const int64_t c_hi = min(hi, a.cl);
    if (c_hi > lo) tma_bulk_g2s(dst, a.carry + lo, static_cast<uint32_t>(c_hi - lo) * 4u, bar);
    const int64_t b_lo = max(lo, a.cl);
    if (hi > b_lo)
        tma_bulk_g2s(dst + (b_lo - lo), a.buf + (b_lo - a.cl), static_cast<uint32_t>(hi - b_lo) * 4u, bar);
}

__device__ __forceinline__ void copy_sb_threads(const PfbArgs& a, int64_t q, int64_t need,
                                                uint32_t* dst) {
    const int64_t lo = q * kSB;
    const int64_t hi = min(lo + kSB, need);
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) dst[i - lo] = vload(a, i);
}

// Writes the frame's outputs: full spectrum from registers, then (if tones)
// the spectrum to smem and the tone gather.  All threads call it.
template <int LOG2N>
__device__ __forceinline__ void pfb_outputs(const PfbArgs& a, float2 (&v)[16], float2* xbuf,
                                            int g, int tf, int64_t j, bool valid, int G,
                                            int64_t j0) {
    constexpr int N = 1 << LOG2N;
    constexpr int FSTRIDE = N + N / 16;
    if (a.full && valid) {
        float2* row = a.full + (a.frame_offset + j) * a.full_ld;
#pragma unroll
        for (int i = 0; i < 16; ++i) row[fft_out_index<LOG2N>(tf, i)] = v[i];
    }
    if (a.n_tones > 0) {
        __syncthreads();   // the passes are done reading xbuf
        float2* fb = xbuf + g * FSTRIDE;
#pragma unroll
        for (int i = 0; i < 16; ++i) fb[fpad(fft_out_index<LOG2N>(tf, i))] = v[i];
        __syncthreads();
        const int items = G * a.n_tones;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int s = it / G, gg = it - s * G;
            const int64_t jj = j0 + gg;
            if (jj >= 0 && jj < a.F) {
                const int b = __ldg(a.bins + s);
                a.tones[s * a.tones_ld + a.frame_offset + jj] = xbuf[gg * FSTRIDE + fpad(b)];
            }
        }
    }
}

// ---------------------------------------------------------------- RING
template <int LOG2N, int T>
__global__ void __launch_bounds__(kRingThreads, 1) pfb_ring_kernel(const PfbArgs a) {
    constexpr int N = 1 << LOG2N;
    constexpr int NT = N / 16;                 // threads per frame
    constexpr int G = kRingThreads / NT;       // frames per iteration
    constexpr int HB = (T - 1 + G - 1) / G;    // history super-blocks
    constexpr int FSTRIDE = N + N / 16;
    static_assert(G * N == kSB, "super-block = G frames");

    extern __shared__ __align__(1024) unsigned char smem[];
    const int RS = a.ring_sb;
    uint32_t* ring = reinterpret_cast<uint32_t*>(smem);
    float2* xbuf = reinterpret_cast<float2*>(smem + static_cast<size_t>(RS) * kSB * 4);
    float2* tw = xbuf + G * FSTRIDE;
    uint64_t* bars = reinterpret_cast<uint64_t*>(tw + ((a.tw_count + 1) & ~1));

    const int tid = threadIdx.x;
    const int g = tid / NT, tf = tid % NT;
    const int64_t need = (a.F + T - 1) * static_cast<int64_t>(N);   // v samples used
    const int64_t n_sb = (need + kSB - 1) / kSB;
    const int64_t qa = a.q_lo + static_cast<int64_t>(blockIdx.x) * a.iters_per_cta;
    const int64_t qb = min(a.q_hi, qa + a.iters_per_cta);
    if (qa >= qb) return;
    const int P = RS - HB - 1;                 // super-blocks of look-ahead

    for (int i = tid; i < a.tw_count; i += blockDim.x) tw[i] = __ldg(a.tw + i);
    // taps of the thread's branches p = tf + r*NT
    float hr[T][16];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int r = 0; r < 16; ++r) hr[t][r] = __ldg(a.h + t * N + tf + r * NT);

    // Super-blocks are issued in order from qs; the fill index of super-block
    // q in its slot (q mod RS) is (q - qs) / RS, which gives the phase parity.
    const int64_t qs = max_i64(qa - HB, 0);
    if (a.use_tma) {
        if (tid == 0) {
            for (int s = 0; s < RS; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0) {
            for (int64_t q = qs; q < min_i64(qa + P + 1, n_sb); ++q)
                issue_sb_tma(a, q, need, ring + static_cast<int64_t>(q % RS) * kSB, &bars[q % RS]);
        }
        for (int64_t q = qs; q < qa; ++q)   // history of the first iteration
            if (!mbar_wait(&bars[q % RS], static_cast<uint32_t>(((q - qs) / RS) & 1), a.status)) return;
    } else {
        for (int64_t q = qs; q < qa; ++q)
            copy_sb_threads(a, q, need, ring + static_cast<int64_t>(q % RS) * kSB);
    }
    const int rlen = RS * kSB;

    for (int64_t q = qa; q < qb; ++q) {
        const int slot = static_cast<int>(q % RS);
        if (a.use_tma) {
            if (!mbar_wait(&bars[slot], static_cast<uint32_t>(((q - qs) / RS) & 1), a.status)) return;
        } else {
            __syncthreads();
            copy_sb_threads(a, q, need, ring + static_cast<int64_t>(slot) * kSB);
            __syncthreads();
        }
        const int64_t j0 = q * G - (T - 1);    // first frame of this iteration
        const int64_t j = j0 + g;
        const bool valid = (j >= 0) && (j < a.F);

        // polyphase FIR
        float2 v[16];
        if (valid) {
            int base = static_cast<int>((j * N) % rlen);
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const uint32_t* blk = ring + base + tf;
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const float2 x = iq_to_f2(blk[r * NT]);
                    v[r].x = fmaf(hr[t][r], x.x, v[r].x);
                    v[r].y = fmaf(hr[t][r], x.y, v[r].y);
                }
                base += N;
                if (base >= rlen) base -= rlen;
            }
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = make_float2(0.f, 0.f);
        }
        __syncthreads();   // ring reads of this iteration are done
        if (a.use_tma && tid == 0) {
            const int64_t qn = q + P + 1;
            if (qn < n_sb) issue_sb_tma(a, qn, need, ring + static_cast<int64_t>(qn % RS) * kSB, &bars[qn % RS]);
        }
        float2* fb = xbuf + g * FSTRIDE;
        fft_frame<LOG2N, true>(v, fb, tf, tw);
        pfb_outputs<LOG2N>(a, v, xbuf, g, tf, j, valid, G, j0);
    }
    // Drain: the look-ahead copies issued past this CTA's range were never
    // waited for; wait for them so no bulk copy lands in freed shared memory.
    if (a.use_tma) {
        for (int64_t q = qb; q < min_i64(qb + P + 1, n_sb); ++q)
            if (!mbar_wait(&bars[q % RS], static_cast<uint32_t>(((q - qs) / RS) & 1), a.status)) return;
    }
}

// ---------------------------------------------------------------- TMEM
// N = 4096, T <= 8 (after padding): the FP32 delay line lives in tensor
// memory.  Each sample is converted from int16 once, stored with tcgen05.st
// into the thread's TMEM columns (slot = block mod 8: 8 blocks x 16 complex
// FP32 per thread = the whole 256 KiB of TMEM for 256 threads), and read back
// for every tap with tcgen05.ld.  int16 blocks arrive by 1-D TMA into a small
// staging ring.  The taps are summed in the same order as the other variants
// (t = 0..T-1 from zero), so results are bit-identical to them.
constexpr int kTmemStage = 4;        // staging slots (blocks of 4096 samples)
constexpr int kTmemSlots = 8;        // delay-line blocks held in TMEM
constexpr int kToneGroup = 4;        // output frames per tone group (32 bytes of each tone row)
constexpr int kToneBox = 256;        // tone rows per TMA store box
constexpr int kTonesPerThread = 5;   // tones in shared memory: at most 5 * 256

// Shared memory of the TMEM variant: int16 staging ring, two exchange
// buffers, twiddles; with the tones in shared memory also their bins and the
// tone tile [rows][kToneGroup] (rows = tones rounded up to the store box,
// 1 KiB aligned); then the mbarriers and the TMEM address.
struct TmemLayout {
    size_t xb, tw, bins, tile, bars, total;
};
__host__ __device__ __forceinline__ TmemLayout tmem_layout(int tw_count, int nb) {
    TmemLayout L{};
    L.xb = static_cast<size_t>(kTmemStage) * 4096 * 4;
    L.tw = L.xb + static_cast<size_t>(2) * (4096 + 256) * 8;
    size_t o = L.tw + static_cast<size_t>((tw_count + 1) & ~1) * 8;
    L.bins = o;
    o = (o + static_cast<size_t>(nb) * 4 + 1023) / 1024 * 1024;
    L.tile = o;
    o += static_cast<size_t>((nb + kToneBox - 1) / kToneBox * kToneBox) * kToneGroup * 8;
    L.bars = o;
    L.total = o + kTmemStage * 8 + 16;
    return L;
}

// PRE: each frame's FIR accumulators start from a.pre's row of the frame
// (the first half of a 16-tap FIR, see fir_pre_kernel) instead of zero;
// the next frame's row is loaded while this frame's FFT runs.
template <int T, bool PRE>
__global__ void __launch_bounds__(kRingThreads, 1)
    pfb_tmem_kernel(const PfbArgs a, const __grid_constant__ CUtensorMap tm_tones) {
    constexpr int N = 4096, NT = 256;
    static_assert(T <= kTmemSlots, "delay line fits in TMEM");
    extern __shared__ __align__(1024) unsigned char smem[];
    const int nb_smem = a.nb_smem;
    const TmemLayout lay = tmem_layout(a.tw_count, nb_smem);
    uint32_t* stage = reinterpret_cast<uint32_t*>(smem);
    // two exchange buffers used alternately (frame parity), so consecutive
    // passes and frames need only three barriers per frame
    float2* const xb0 = reinterpret_cast<float2*>(smem + lay.xb);
    float2* const xb1 = xb0 + (N + N / 16);
    float2* tw = reinterpret_cast<float2*>(smem + lay.tw);
    int32_t* sbins = reinterpret_cast<int32_t*>(smem + lay.bins);
    float2* tile = reinterpret_cast<float2*>(smem + lay.tile);   // tone t, group frame q at t*kToneGroup + q
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + lay.bars);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + kTmemStage);

    const int tid = threadIdx.x, warp = tid >> 5, tf = tid;
    // CTA ranges start on whole tone groups of OUTPUT frames (frame_offset + j
    // a multiple of kToneGroup), so every TMA store origin is 32-byte aligned
    const int64_t shift = a.frame_offset & (kToneGroup - 1);
    const int64_t ja = max_i64(0, static_cast<int64_t>(blockIdx.x) * a.iters_per_cta - shift);
    const int64_t jb = min_i64(a.F, static_cast<int64_t>(blockIdx.x + 1) * a.iters_per_cta - shift);
    if (ja >= jb) return;
    const int64_t b0 = ja, b1 = jb + T - 1;                     // blocks [b0, b1)
    const int64_t need = (a.F + T - 1) * static_cast<int64_t>(N);

    if (warp == 0) {
        umma::alloc(tmem_holder, 512);
        umma::relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kTmemStage; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    for (int i = tid; i < a.tw_count; i += blockDim.x) tw[i] = __ldg(a.tw + i);
    for (int i = tid; i < nb_smem; i += blockDim.x) sbins[i] = __ldg(a.bins + i);
    float hr[T][16];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int r = 0; r < 16; ++r) hr[t][r] = __ldg(a.h + t * N + tf + r * NT);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tbase = *tmem_holder + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                           static_cast<uint32_t>(256 * (warp >> 2));
    if (tid == 0)
        for (int64_t b = b0; b < min_i64(b0 + kTmemStage, b1); ++b)
            issue_sb_tma(a, b, need, stage + (b % kTmemStage) * N, &bars[b % kTmemStage]);

    bool ok = true;
    float are[16], aim[16];
    bool pre_loaded = false;
    auto load_pre = [&](int64_t jj) {
        const float2* row = a.pre + jj * N + tf;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const float2 q = __ldg(row + r * NT);
            are[r] = q.x;
            aim[r] = q.y;
        }
    };
    for (int64_t b = b0; b < b1; ++b) {
        const int s = static_cast<int>(b % kTmemStage);
        if (!mbar_wait(&bars[s], static_cast<uint32_t>(((b - b0) / kTmemStage) & 1), a.status)) {
            ok = false;
            break;
        }
        // planar pairs in TMEM: (re_r, re_r+1, im_r, im_r+1) for even r
        uint32_t xr[32];
#pragma unroll
        for (int r = 0; r < 16; r += 2) {
            const float2 f0 = iq_to_f2(stage[s * N + tf + r * NT]);
            const float2 f1 = iq_to_f2(stage[s * N + tf + (r + 1) * NT]);
            xr[2 * r] = __float_as_uint(f0.x);
            xr[2 * r + 1] = __float_as_uint(f1.x);
            xr[2 * r + 2] = __float_as_uint(f0.y);
            xr[2 * r + 3] = __float_as_uint(f1.y);
        }
        umma::st_32x32b_x32(tbase + 32u * static_cast<uint32_t>(b % kTmemSlots), xr);
        umma::wait_st();
        const int64_t j = b - (T - 1);                           // frame completed by block b
        if (j < ja) {                                            // uniform across the CTA
            __syncthreads();                                     // staging slot s fully read
            if (tid == 0 && b + kTmemStage < b1)
                issue_sb_tma(a, b + kTmemStage, need, stage + s * N, &bars[s]);
            continue;
        }
        if constexpr (PRE) {
            if (!pre_loaded) load_pre(j);                        // the CTA's first frame
            pre_loaded = false;
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) are[r] = aim[r] = 0.f;
        }
        // taps in order t = 0..T-1; each slot read as two 16-column halves,
        // the next half's load in flight while this half's FMAs issue
        uint32_t xa[16], xb[16];
        umma::ld_32x32b_x16(tbase + 32u * static_cast<uint32_t>(j % kTmemSlots), xa);
        umma::wait_ld_regs(xa);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint32_t col = tbase + 32u * static_cast<uint32_t>((j + t) % kTmemSlots);
            umma::ld_32x32b_x16(col + 16u, xb);
#pragma unroll
            for (int r = 0; r < 8; r += 2) {
                ffma2(are[r], are[r + 1], hr[t][r], hr[t][r + 1], __uint_as_float(xa[2 * r]),
                      __uint_as_float(xa[2 * r + 1]));
                ffma2(aim[r], aim[r + 1], hr[t][r], hr[t][r + 1], __uint_as_float(xa[2 * r + 2]),
                      __uint_as_float(xa[2 * r + 3]));
            }
            umma::wait_ld_regs(xb);
            if (t + 1 < T)
                umma::ld_32x32b_x16(tbase + 32u * static_cast<uint32_t>((j + t + 1) % kTmemSlots), xa);
#pragma unroll
            for (int r = 8; r < 16; r += 2) {
                ffma2(are[r], are[r + 1], hr[t][r], hr[t][r + 1], __uint_as_float(xb[2 * r - 16]),
                      __uint_as_float(xb[2 * r - 15]));
                ffma2(aim[r], aim[r + 1], hr[t][r], hr[t][r + 1], __uint_as_float(xb[2 * r - 14]),
                      __uint_as_float(xb[2 * r - 13]));
            }
            if (t + 1 < T) umma::wait_ld_regs(xa);
        }
        float2 v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = make_float2(are[r], aim[r]);
        if constexpr (PRE) {
            if (j + 1 < jb) {
                load_pre(j + 1);
                pre_loaded = true;
            }
        }
        // 4096-point Stockham FFT, 3 radix-16 passes (as fft_frame<12>):
        // pass 0 -> P, pass 1 P -> Q, pass 2 Q -> registers; spectrum -> P.
        float2* const P = (j & 1) ? xb1 : xb0;
        float2* const Q = (j & 1) ? xb0 : xb1;
        dft16(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) P[fpad(16 * tf + r)] = v[r];
        // the previous frame's bulk stores have read the spectrum row (now Q's
        // twin) and the tone tile before either is written again
        if (tid == 0) bulk_wait_read_all();
        __syncthreads();                                         // (A) pass 0 written, staging read
        if (tid == 0 && b + kTmemStage < b1)
            issue_sb_tma(a, b + kTmemStage, need, stage + s * N, &bars[s]);
        {
            const int k = tf & 15;
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = P[fpad(tf + r * NT)];
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw[(r - 1) * 16 + k]);
            dft16(v);
            const int base = (tf >> 4) * 256 + k;
#pragma unroll
            for (int r = 0; r < 16; ++r) Q[fpad(base + r * 16)] = v[r];
        }
        __syncthreads();                                         // (B) pass 1 written
        {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = Q[fpad(tf + r * NT)];
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw[240 + (r - 1) * 256 + tf]);
            dft16(v);                                            // v[r] = bin tf + 256 r
        }
        // Outputs.  The spectrum goes to P (unpadded natural order when the
        // full row leaves by one bulk store, padded when only the tones read
        // it).  Tones in shared memory: thread tid gathers tones tid + 256 k
        // into the tone tile (all bins, then all values, then all stores, so
        // the loads overlap); a group of kToneGroup output frames leaves by
        // 2-D TMA stores (whole groups) or plain stores (a CTA's partial
        // first or last group, unaligned rows).  More tones: each is gathered
        // from P and stored per frame.
        const bool bulk = a.full_bulk != 0;
        if (a.full && !bulk) {
            float2* row = a.full + (a.frame_offset + j) * a.full_ld;
#pragma unroll
            for (int i = 0; i < 16; ++i) row[tf + i * NT] = v[i];
        }
        if (bulk) {
#pragma unroll
            for (int i = 0; i < 16; ++i) P[tf + i * NT] = v[i];
            fence_proxy_async_smem();
        } else if (a.n_tones > 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) P[fpad(tf + i * NT)] = v[i];
        }
        __syncthreads();                                         // (C) spectrum in P; Q reads done
        if (bulk && tid == 0) {
            tma_bulk_s2g(a.full + (a.frame_offset + j) * a.full_ld, P, N * 8);
            bulk_commit();
        }
        if (nb_smem > 0) {
            const int q = static_cast<int>((a.frame_offset + j) & (kToneGroup - 1));
            int bk[kTonesPerThread];
#pragma unroll
            for (int k = 0; k < kTonesPerThread; ++k) bk[k] = tid + k * NT < nb_smem ? sbins[tid + k * NT] : -1;
            float2 tv[kTonesPerThread];
#pragma unroll
            for (int k = 0; k < kTonesPerThread; ++k)
                if (bk[k] >= 0) tv[k] = P[bulk ? bk[k] : fpad(bk[k])];
#pragma unroll
            for (int k = 0; k < kTonesPerThread; ++k)
                if (bk[k] >= 0) tile[(tid + k * NT) * kToneGroup + q] = tv[k];
            if (q == kToneGroup - 1 || j == jb - 1) {
                const bool gtma = a.tones_tma && q == kToneGroup - 1 && j - q >= ja;
                if (gtma) fence_proxy_async_smem();
                __syncthreads();                                 // tile complete
                if (gtma) {
                    if (tid == 0) {
                        const int32_t x0 = static_cast<int32_t>(a.frame_offset + j - q);
                        for (int r0 = 0; r0 < nb_smem; r0 += kToneBox)
                            tma_store_2d(&tm_tones, x0, r0, tile + static_cast<size_t>(r0) * kToneGroup);
                        bulk_commit();
                    }
                } else {
                    // frames j - q .. j of the group that this CTA produced
                    const int q0 = static_cast<int>(max_i64(0, ja - (j - q)));
                    const int nq = q + 1 - q0;
                    float2* base = a.tones + a.frame_offset + (j - q);
                    for (int it = tid; it < nq * nb_smem; it += NT) {
                        const int t = it / nq, qq = q0 + (it - t * nq);
                        base[static_cast<int64_t>(t) * a.tones_ld + qq] = tile[t * kToneGroup + qq];
                    }
                }
            }
        } else if (a.n_tones > 0) {
            float2* col = a.tones + a.frame_offset + j;
            for (int t = tid; t < a.n_tones; t += NT) {
                const int bin = __ldg(a.bins + t);
                col[t * a.tones_ld] = P[bulk ? bin : fpad(bin)];
            }
        }
    }
    if (tid == 0) bulk_wait_all();
    (void)ok;
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after_sync();
        umma::dealloc(*tmem_holder, 512);
    }
}

// ------------------------------------------------- TMEM, symmetric taps
// N = 4096, T = 8 with an exactly symmetric prototype, h[j] = h[8N - 1 - j]
// (the plan builds it so).  Same stream view, TMEM delay line, sum order
// and outputs as pfb_tmem_kernel (bit-identical results), arranged so that
// a frame costs two CTA barriers instead of three and no twiddle traffic
// through shared memory:
//   - Lanes l and 31 - l of a warp own the mirrored FFT rows tf and 255 - tf
//     (row tf = the points tf + 256 r).  A thread filters its row's points
//     r < 8 and the mirror points (255 - tf, 15 - r), whose taps are the same
//     values in reverse tap order, so it holds 64 tap registers instead of
//     128; one warp shuffle per value then swaps the mirrored halves so that
//     every thread has its whole row for the first radix-16 pass.
//   - The 2 x 15 twiddles of passes 1 and 2 depend only on the row: they
//     live in registers.
//   - Three exchange buffers: pass 0 writes B0, pass 1 B1, pass 2 writes the
//     spectrum to B2 (natural order).  The spectrum of frame j is stored (TMA
//     bulk) and its tones gathered while pass 1 of frame j + 1 runs, so the
//     iteration has one barrier after pass 0 and one after pass 1.
constexpr size_t kSymXb = static_cast<size_t>(4096 + 256) * 8;
struct SymLayout {
    size_t b0, b1, b2, bins, tile, bars, total;
};
__host__ __device__ __forceinline__ SymLayout sym_layout(int nb) {
    SymLayout L{};
    L.b0 = static_cast<size_t>(kTmemStage) * 4096 * 4;
    L.b1 = L.b0 + kSymXb;
    L.b2 = L.b1 + kSymXb;
    size_t o = L.b2 + static_cast<size_t>(4096) * 8;
    L.bins = o;
    o = (o + static_cast<size_t>(nb) * 4 + 1023) / 1024 * 1024;
    L.tile = o;
    o += static_cast<size_t>((nb + kToneBox - 1) / kToneBox * kToneBox) * kToneGroup * 8;
    L.bars = o;
    L.total = o + kTmemStage * 8 + 16;
    return L;
}

template <bool PHASE>
__global__ void __launch_bounds__(kRingThreads, 1)
    pfb_tmem_sym_kernel(const PfbArgs a, const __grid_constant__ CUtensorMap tm_tones) {
    constexpr int N = 4096, NT = 256, T = 8;
    // PHASE: a phase pass of an oversampled plan (tone columns a.tone_cs
    // apart, bins turned by (-i)^(c * a.rot)); otherwise adjacent columns, no turn
    const int64_t tcs = PHASE ? a.tone_cs : 1;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int nb_smem = a.nb_smem;
    const SymLayout lay = sym_layout(nb_smem);
    uint32_t* stage = reinterpret_cast<uint32_t*>(smem);
    float2* const B0 = reinterpret_cast<float2*>(smem + lay.b0);
    float2* const B1 = reinterpret_cast<float2*>(smem + lay.b1);
    float2* const B2 = reinterpret_cast<float2*>(smem + lay.b2);
    int32_t* sbins = reinterpret_cast<int32_t*>(smem + lay.bins);
    float2* tile = reinterpret_cast<float2*>(smem + lay.tile);   // tone t, group frame q at t*kToneGroup + q
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + lay.bars);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + kTmemStage);
    volatile int* s_ok = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tf = lane < 16 ? 16 * warp + lane : 224 - 16 * warp + lane;   // partner lane 31 - l: 255 - tf
    const int64_t shift = a.frame_offset & (kToneGroup - 1);
    const int64_t ja = max_i64(0, static_cast<int64_t>(blockIdx.x) * a.iters_per_cta - shift);
    const int64_t jb = min_i64(a.F, static_cast<int64_t>(blockIdx.x + 1) * a.iters_per_cta - shift);
    if (ja >= jb) return;
    const int64_t b0 = ja, b1 = jb + T - 1;                     // blocks [b0, b1)
    const int64_t need = (a.F + T - 1) * static_cast<int64_t>(N);

    if (warp == 0) {
        umma::alloc(tmem_holder, 512);
        umma::relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kTmemStage; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    for (int i = tid; i < nb_smem; i += blockDim.x) sbins[i] = __ldg(a.bins + i);
    // taps of the own points (tf, q), q < 8; the mirror point (255-tf, 15-q)
    // takes tap t from H[T-1-t][q]
    float H[T][8];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int q = 0; q < 8; ++q) H[t][q] = __ldg(a.h + t * N + tf + q * NT);
    float2 w1[15], w2[15];
    {
        const int k = tf & 15;
#pragma unroll
        for (int r = 1; r < 16; ++r) {
            w1[r - 1] = __ldg(a.tw + (r - 1) * 16 + k);
            w2[r - 1] = __ldg(a.tw + 240 + (r - 1) * 256 + tf);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tbase = *tmem_holder + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                           static_cast<uint32_t>(256 * (warp >> 2));
    if (tid == 0)
        for (int64_t b = b0; b < min_i64(b0 + kTmemStage, b1); ++b)
            issue_sb_tma(a, b, need, stage + (b % kTmemStage) * N, &bars[b % kTmemStage]);

    // int16 block b (staging slot s) -> FP32 -> the thread's TMEM columns of
    // slot b mod 8: points (tf, q) then the mirror points (255-tf, 15-m), as
    // planar pairs (re_q, re_q+1, im_q, im_q+1)
    auto ingest = [&](int64_t b, int s) {
        // the phase completed already (thread 0 saw it before the last
        // barrier); each thread's own wait makes the copy visible to it
        mbar_wait(&bars[s], static_cast<uint32_t>(((b - b0) / kTmemStage) & 1), a.status);
        uint32_t xr[32];
        const uint32_t* sg = stage + s * N;
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
            const int p0 = q < 8 ? tf + q * NT : 4095 - tf - (q - 8) * NT;
            const int p1 = q < 8 ? tf + (q + 1) * NT : 4095 - tf - (q - 7) * NT;
            const float2 f0 = iq_to_f2(sg[p0]);
            const float2 f1 = iq_to_f2(sg[p1]);
            xr[2 * q] = __float_as_uint(f0.x);
            xr[2 * q + 1] = __float_as_uint(f1.x);
            xr[2 * q + 2] = __float_as_uint(f0.y);
            xr[2 * q + 3] = __float_as_uint(f1.y);
        }
        umma::st_32x32b_x32(tbase + 32u * static_cast<uint32_t>(b % kTmemSlots), xr);
        umma::wait_st();
    };
    auto stage_parity = [&](int64_t b) { return static_cast<uint32_t>(((b - b0) / kTmemStage) & 1); };

    // warm-up: the T - 1 blocks before the first frame's last one
    bool ok = true;
    for (int64_t b = b0; b < b0 + T - 1; ++b) {
        const int s = static_cast<int>(b % kTmemStage);
        const bool got = mbar_wait(&bars[s], stage_parity(b), a.status);
        if (__syncthreads_or(!got)) {
            ok = false;
            break;
        }
        ingest(b, s);
        __syncthreads();                                         // staging slot s read by all
        if (tid == 0 && b + kTmemStage < b1)
            issue_sb_tma(a, b + kTmemStage, need, stage + s * N, &bars[s]);
    }
    if (ok) {
        if (tid == 0) *s_ok = mbar_wait(&bars[(b0 + T - 1) % kTmemStage], stage_parity(b0 + T - 1), a.status) ? 1 : 0;
        __syncthreads();
        ok = *s_ok != 0;
    }
    const bool bulk = a.full_bulk != 0;
    int64_t jp = -1;                                             // frame whose spectrum is in B2
    // stores and gathers the spectrum of frame jp (in B2) into the tone tile
    auto gather = [&](int64_t j) {
        if (bulk && tid == 0) {
            tma_bulk_s2g(a.full + (a.frame_offset + j) * a.full_ld, B2, N * 8);
            bulk_commit();
        }
        if (nb_smem > 0) {
            const int q = static_cast<int>((a.frame_offset + j) & (kToneGroup - 1));
            int bk[kTonesPerThread];
#pragma unroll
            for (int k = 0; k < kTonesPerThread; ++k) bk[k] = tid + k * NT < nb_smem ? sbins[tid + k * NT] : -1;
            float2 tv[kTonesPerThread];
#pragma unroll
            for (int k = 0; k < kTonesPerThread; ++k)
                if (bk[k] >= 0) tv[k] = B2[bk[k]];
#pragma unroll
            for (int k = 0; k < kTonesPerThread; ++k)
                if (bk[k] >= 0) tile[(tid + k * NT) * kToneGroup + q] = tv[k];
        } else if (a.n_tones > 0) {
            float2* col = a.tones + (a.frame_offset + j) * tcs;
            for (int t = tid; t < a.n_tones; t += NT) col[t * a.tones_ld] = B2[__ldg(a.bins + t)];
        }
    };
    // group of frame j complete (last of a tone group or of the CTA's range)?
    auto closes_group = [&](int64_t j) {
        return nb_smem > 0 && ((((a.frame_offset + j) & (kToneGroup - 1)) == kToneGroup - 1) || j == jb - 1);
    };
    auto tile_by_tma = [&](int64_t j) {
        const int q = static_cast<int>((a.frame_offset + j) & (kToneGroup - 1));
        return a.tones_tma && q == kToneGroup - 1 && j - q >= ja;
    };
    // writes the tone group that frame j closed (after a barrier that
    // follows every thread's gather)
    auto flush_group = [&](int64_t j) {
        const int q = static_cast<int>((a.frame_offset + j) & (kToneGroup - 1));
        if (tile_by_tma(j)) {
            if (tid == 0) {
                const int32_t x0 = static_cast<int32_t>(a.frame_offset + j - q);
                for (int r0 = 0; r0 < nb_smem; r0 += kToneBox)
                    tma_store_2d(&tm_tones, x0, r0, tile + static_cast<size_t>(r0) * kToneGroup);
                bulk_commit();
            }
        } else {
            // frames j - q .. j of the group that this CTA produced
            const int q0 = static_cast<int>(max_i64(0, ja - (j - q)));
            const int nq = q + 1 - q0;
            float2* base = a.tones + (a.frame_offset + (j - q)) * tcs;
            for (int it = tid; it < nq * nb_smem; it += NT) {
                const int t = it / nq, qq = q0 + (it - t * nq);
                base[static_cast<int64_t>(t) * a.tones_ld + qq * tcs] = tile[t * kToneGroup + qq];
            }
        }
    };

    for (int64_t j = ja; ok && j < jb; ++j) {
        const int64_t b = j + T - 1;                             // the block that completes frame j
        const int s = static_cast<int>(b % kTmemStage);
        ingest(b, s);
        // polyphase FIR, taps in order t = 0..T-1 (slot halves: own points,
        // then mirror points, the next load in flight during the FMAs)
        float are[16], aim[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) are[r] = aim[r] = 0.f;
        uint32_t xa[16], xb[16];
        umma::ld_32x32b_x16(tbase + 32u * static_cast<uint32_t>(j % kTmemSlots), xa);
        umma::wait_ld_regs(xa);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint32_t col = tbase + 32u * static_cast<uint32_t>((j + t) % kTmemSlots);
            umma::ld_32x32b_x16(col + 16u, xb);
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                ffma2(are[q], are[q + 1], H[t][q], H[t][q + 1], __uint_as_float(xa[2 * q]),
                      __uint_as_float(xa[2 * q + 1]));
                ffma2(aim[q], aim[q + 1], H[t][q], H[t][q + 1], __uint_as_float(xa[2 * q + 2]),
                      __uint_as_float(xa[2 * q + 3]));
            }
            umma::wait_ld_regs(xb);
            if (t + 1 < T)
                umma::ld_32x32b_x16(tbase + 32u * static_cast<uint32_t>((j + t + 1) % kTmemSlots), xa);
#pragma unroll
            for (int m = 0; m < 8; m += 2) {
                ffma2(are[8 + m], are[9 + m], H[T - 1 - t][m], H[T - 1 - t][m + 1], __uint_as_float(xb[2 * m]),
                      __uint_as_float(xb[2 * m + 1]));
                ffma2(aim[8 + m], aim[9 + m], H[T - 1 - t][m], H[T - 1 - t][m + 1],
                      __uint_as_float(xb[2 * m + 2]), __uint_as_float(xb[2 * m + 3]));
            }
            if (t + 1 < T) umma::wait_ld_regs(xa);
        }
        // the partner (lane 31 - l) filtered this row's points 8..15
        float2 v[16];
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = make_float2(are[r], aim[r]);
#pragma unroll
        for (int m = 0; m < 8; ++m)
            v[15 - m] = make_float2(__shfl_xor_sync(0xffffffffu, are[8 + m], 31),
                                    __shfl_xor_sync(0xffffffffu, aim[8 + m], 31));
        // pass 0 -> B0
        dft16(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) B0[fpad(16 * tf + r)] = v[r];
        if (tid == 0) bulk_wait_read_all();                     // tile stores done reading the tile
        __syncthreads();                                         // (1) B0 written, staging slot s read
        if (tid == 0 && b + kTmemStage < b1)
            issue_sb_tma(a, b + kTmemStage, need, stage + s * N, &bars[s]);
        // outputs of the previous frame while pass 1 of this one runs
        if (jp >= 0) gather(jp);
        {
            const int k = tf & 15;
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = B0[fpad(tf + r * NT)];
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], w1[r - 1]);
            dft16(v);
            const int base = (tf >> 4) * 256 + k;
#pragma unroll
            for (int r = 0; r < 16; ++r) B1[fpad(base + r * 16)] = v[r];
        }
        const bool close_prev = jp >= 0 && closes_group(jp);
        if (close_prev && tile_by_tma(jp)) fence_proxy_async_smem();
        if (tid == 0) {
            bulk_wait_read_all();                                // B2 read by its row store
            *s_ok = (j + 1 < jb) ? (mbar_wait(&bars[(b + 1) % kTmemStage], stage_parity(b + 1), a.status) ? 1 : 0) : 1;
        }
        __syncthreads();                                         // (2) B1 written, gathers done
        if (close_prev) flush_group(jp);
        {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = B1[fpad(tf + r * NT)];
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], w2[r - 1]);
            dft16(v);                                            // v[r] = bin tf + 256 r
        }
        if (PHASE && a.rot) {
            // (-i)^e, e = (c * rot) mod 4 for c = tf + 256 r: the same power for
            // all r, and it differs between the lanes of a warp, so it is applied
            // without branches: odd e swaps re and im, then sign bits are flipped
            // (e = 1: (im, -re); 2: (-re, -im); 3: (-im, re)); exact
            const int e = (tf * a.rot) & 3;
            const bool sw = (e & 1) != 0;
            const uint32_t m_re = (e == 2 || e == 3) ? 0x80000000u : 0u;
            const uint32_t m_im = (e == 1 || e == 2) ? 0x80000000u : 0u;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float2 u = v[i];
                const float re = sw ? u.y : u.x, im = sw ? u.x : u.y;
                v[i] = make_float2(__uint_as_float(__float_as_uint(re) ^ m_re), __uint_as_float(__float_as_uint(im) ^ m_im));
            }
        }
        if (a.full && !bulk) {
            float2* row = a.full + (a.frame_offset + j) * a.full_ld;
#pragma unroll
            for (int i = 0; i < 16; ++i) row[tf + i * NT] = v[i];
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) B2[tf + i * NT] = v[i];
        fence_proxy_async_smem();
        jp = j;
        ok = *s_ok != 0;
    }
    if (ok && jp >= 0) {
        if (tid == 0) bulk_wait_read_all();                     // tile stores done reading the tile
        __syncthreads();                                         // spectrum of the last frame in B2
        gather(jp);
        if (closes_group(jp)) {
            if (tile_by_tma(jp)) fence_proxy_async_smem();
            __syncthreads();
            flush_group(jp);
        }
    }
    if (tid == 0) bulk_wait_all();
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after_sync();
        umma::dealloc(*tmem_holder, 512);
    }
}

// ------------------------------------------------- CLUSTER (N = 8192, 16384)
// N = C * 4096 channels (C = 2 or 4), T <= 8 taps: the FP32 delay line of
// N * T points exceeds one SM's tensor memory, so a cluster of C CTAs on C
// SMs shares every frame.  CTA c (its rank in the cluster) owns channels
// [4096 c, 4096 c + 4096): their staging, delay line in TMEM and taps in
// registers, exactly as the one-SM kernel above.  The N-point DFT of the
// filtered frame v is split as p = 4096 c + p1, k = k2 + C k1:
//   y[k2 + C k1] = sum_p1 W_4096^(k1 p1) * W_N^(k2 p1) * sum_c W_C^(k2 c) v[4096 c + p1],
// so after the FIR each CTA puts its slice in shared memory (E), the
// cluster meets (S1), CTA k2 forms u[p1] = W_N^(k2 p1) sum_c W_C^(k2 c) E_c[p1]
// from the C slices (distributed shared memory reads; W_C^m is an exact
// quarter-turn power or a sign), runs the 4096-point FFT of the one-SM
// kernel on u and leaves bins k2 + C k1 in its buffer P; the cluster meets
// again (S2) and CTA c assembles output bins [4096 c, 4096 c + 4096) from
// the C buffers into one contiguous row piece (one TMA bulk store) and
// gathers its share of the tones (a contiguous range of tone rows, whole
// 256-row boxes) the same way.  Waits on the staging ring are bounded; a
// CTA whose wait gave up keeps taking part in every cluster barrier (with
// no further copies) so that no peer is left waiting.  A plan choice
// (rfr_plan_set_pfb_cluster), not the default: with one frame in flight per
// CTA the exchanges and the two cluster barriers of every frame stay
// exposed, and the direct kernel measured faster.
constexpr int kClusterTonesPerCta = kTonesPerThread * kRingThreads;
struct ClusterLayout {
    size_t xb, tw, bins, tile, bars, total;
};
__host__ __device__ __forceinline__ ClusterLayout cluster_layout(int tw_count, int nb) {
    ClusterLayout L{};
    L.xb = static_cast<size_t>(kTmemStage) * 4096 * 4;
    L.tw = L.xb + static_cast<size_t>(3) * (4096 + 256) * 8;             // P / Q pair and E
    size_t o = L.tw + static_cast<size_t>(((tw_count + 1) & ~1) + 16) * 8;  // + W_N^(k2 256 r), r < 16
    L.bins = o;
    o = (o + static_cast<size_t>(nb) * 4 + 1023) / 1024 * 1024;
    L.tile = o;
    o += static_cast<size_t>((nb + kToneBox - 1) / kToneBox * kToneBox) * kToneGroup * 8;
    L.bars = o;
    L.total = o + kTmemStage * 8 + 16;
    return L;
}

// Address of `p` (this CTA's shared memory) in cluster CTA `rank`.
__device__ __forceinline__ uint32_t dsmem_map(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 dsmem_ld_f2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
// z * (-i)^m, exact
__device__ __forceinline__ float2 quarter_turn(float2 z, int m) {
    switch (m & 3) {
    case 0: return z;
    case 1: return make_float2(z.y, -z.x);
    case 2: return make_float2(-z.x, -z.y);
    default: return make_float2(-z.y, z.x);
    }
}

// a.tw: the 4096-point FFT twiddles (a.tw_count entries), then W_N^(k2 p1)
// at a.tw + a.tw_count + k2 * 4096 + p1.  a.nb_smem: tones per CTA (a
// multiple of kToneBox, or 0: tones gathered per frame without the tile).
template <int C, int T>
__global__ void __launch_bounds__(kRingThreads, 1)
    pfb_cluster_kernel(const PfbArgs a, const __grid_constant__ CUtensorMap tm_tones) {
    constexpr int NB = 4096, NT = 256, N = C * NB;
    static_assert(C == 2 || C == 4, "cluster of 2 or 4 CTAs");
    static_assert(T <= kTmemSlots, "delay line fits in TMEM");
    constexpr int XS = NB + NB / 16;                              // padded buffer length
    extern __shared__ __align__(1024) unsigned char smem[];
    const int ntc = a.nb_smem;                                    // tone rows per CTA
    const ClusterLayout lay = cluster_layout(a.tw_count, ntc);
    uint32_t* stage = reinterpret_cast<uint32_t*>(smem);
    float2* const xb0 = reinterpret_cast<float2*>(smem + lay.xb);
    float2* const xb1 = xb0 + XS;
    float2* const E = xb1 + XS;
    float2* tw = reinterpret_cast<float2*>(smem + lay.tw);
    int32_t* sbins = reinterpret_cast<int32_t*>(smem + lay.bins);
    float2* tile = reinterpret_cast<float2*>(smem + lay.tile);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + lay.bars);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + kTmemStage);

    const int tid = threadIdx.x, warp = tid >> 5, tf = tid;
    const int rank = static_cast<int>(cluster_ctarank());
    const int64_t cid = blockIdx.x / C;
    // frames [ja, jb) of this cluster (the same for its C CTAs), whole tone
    // groups of output frames as in the one-SM kernel
    const int64_t shift = a.frame_offset & (kToneGroup - 1);
    const int64_t ja = max_i64(0, cid * a.iters_per_cta - shift);
    const int64_t jb = min_i64(a.F, (cid + 1) * a.iters_per_cta - shift);
    if (ja >= jb) return;                                         // the whole cluster returns
    const int64_t b0 = ja, b1 = jb + T - 1;
    const int64_t need = (a.F + T - 1) * static_cast<int64_t>(N);
    // this CTA's tone rows [t0, t1)
    const int t0 = ntc > 0 ? min(a.n_tones, rank * ntc) : (a.n_tones * rank) / C;
    const int t1 = ntc > 0 ? min(a.n_tones, t0 + ntc) : (a.n_tones * (rank + 1)) / C;

    if (warp == 0) {
        umma::alloc(tmem_holder, 512);
        umma::relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kTmemStage; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    for (int i = tid; i < a.tw_count; i += blockDim.x) tw[i] = __ldg(a.tw + i);
    // cross twiddles W_N^(rank p1), p1 = tf + 256 r, as W_N^(rank tf) (a
    // register) times W_N^(rank 256 r) (16 values in shared memory)
    float2* const xtw_r = tw + ((a.tw_count + 1) & ~1);
    if (tid < 16) xtw_r[tid] = __ldg(a.tw + a.tw_count + rank * NB + tid * NT);
    const float2 xtw_t = __ldg(a.tw + a.tw_count + rank * NB + tf);
    if (ntc > 0)
        for (int i = tid; i < t1 - t0; i += blockDim.x) sbins[i] = __ldg(a.bins + t0 + i);
    float hr[T][16];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int r = 0; r < 16; ++r) hr[t][r] = __ldg(a.h + t * N + rank * NB + tf + r * NT);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    cluster_sync();                                               // every peer is running
    const uint32_t tbase = *tmem_holder + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                           static_cast<uint32_t>(256 * (warp >> 2));
    const bool tma = a.use_tma != 0;
    if (tma && tid == 0)
        for (int64_t b = b0; b < min_i64(b0 + kTmemStage, b1); ++b)
            issue_sb_tma(a, b * C + rank, need, stage + (b % kTmemStage) * NB, &bars[b % kTmemStage]);

    bool ok = true;
    for (int64_t b = b0; b < b1; ++b) {
        const int s = static_cast<int>(b % kTmemStage);
        if (tma) {
            if (ok && !mbar_wait(&bars[s], static_cast<uint32_t>(((b - b0) / kTmemStage) & 1), a.status)) ok = false;
        } else {
            copy_sb_threads(a, b * C + rank, need, stage + s * NB);
            __syncthreads();
        }
        uint32_t xr[32];
#pragma unroll
        for (int r = 0; r < 16; r += 2) {
            const float2 f0 = iq_to_f2(stage[s * NB + tf + r * NT]);
            const float2 f1 = iq_to_f2(stage[s * NB + tf + (r + 1) * NT]);
            xr[2 * r] = __float_as_uint(f0.x);
            xr[2 * r + 1] = __float_as_uint(f1.x);
            xr[2 * r + 2] = __float_as_uint(f0.y);
            xr[2 * r + 3] = __float_as_uint(f1.y);
        }
        umma::st_32x32b_x32(tbase + 32u * static_cast<uint32_t>(b % kTmemSlots), xr);
        umma::wait_st();
        const int64_t j = b - (T - 1);
        if (j < ja) {                                             // uniform across the cluster
            __syncthreads();                                      // staging slot s fully read
            if (tma && ok && tid == 0 && b + kTmemStage < b1)
                issue_sb_tma(a, (b + kTmemStage) * C + rank, need, stage + s * NB, &bars[s]);
            continue;
        }
        // FIR of this CTA's 4096 channels (taps t = 0..T-1 in order)
        float are[16], aim[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) are[r] = aim[r] = 0.f;
        uint32_t xa[16], xb[16];
        umma::ld_32x32b_x16(tbase + 32u * static_cast<uint32_t>(j % kTmemSlots), xa);
        umma::wait_ld_regs(xa);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint32_t col = tbase + 32u * static_cast<uint32_t>((j + t) % kTmemSlots);
            umma::ld_32x32b_x16(col + 16u, xb);
#pragma unroll
            for (int r = 0; r < 8; r += 2) {
                ffma2(are[r], are[r + 1], hr[t][r], hr[t][r + 1], __uint_as_float(xa[2 * r]),
                      __uint_as_float(xa[2 * r + 1]));
                ffma2(aim[r], aim[r + 1], hr[t][r], hr[t][r + 1], __uint_as_float(xa[2 * r + 2]),
                      __uint_as_float(xa[2 * r + 3]));
            }
            umma::wait_ld_regs(xb);
            if (t + 1 < T)
                umma::ld_32x32b_x16(tbase + 32u * static_cast<uint32_t>((j + t + 1) % kTmemSlots), xa);
#pragma unroll
            for (int r = 8; r < 16; r += 2) {
                ffma2(are[r], are[r + 1], hr[t][r], hr[t][r + 1], __uint_as_float(xb[2 * r - 16]),
                      __uint_as_float(xb[2 * r - 15]));
                ffma2(aim[r], aim[r + 1], hr[t][r], hr[t][r + 1], __uint_as_float(xb[2 * r - 14]),
                      __uint_as_float(xb[2 * r - 13]));
            }
            if (t + 1 < T) umma::wait_ld_regs(xa);
        }
#pragma unroll
        for (int r = 0; r < 16; ++r) E[fpad(tf + r * NT)] = make_float2(are[r], aim[r]);
        // the previous frame's row piece (in this frame's P) and tone tile
        // have been read by their bulk stores before either is written again
        if (tid == 0) bulk_wait_read_all();
        cluster_sync();                                           // (S1) every slice in E; staging read
        if (tma && ok && tid == 0 && b + kTmemStage < b1)
            issue_sb_tma(a, (b + kTmemStage) * C + rank, need, stage + s * NB, &bars[s]);
        // u[p1] = W_N^(rank p1) * sum_c W_C^(rank c) E_c[p1], p1 = tf + 256 r
        // (the cross twiddles of k2 = rank follow the FFT twiddles in a.tw)
        float2 v[16];
        {
            uint32_t e_at[C];                                     // E of each cluster CTA
#pragma unroll
            for (int c = 0; c < C; ++c) e_at[c] = dsmem_map(E, static_cast<uint32_t>(c)) + static_cast<uint32_t>(fpad(tf)) * 8u;
            // remote loads issued in groups of 16 before their first use, so
            // their latencies overlap
            constexpr int RG = 16 / C;                            // points per group
#pragma unroll
            for (int r0 = 0; r0 < 16; r0 += RG) {
                float2 e[RG][C];
#pragma unroll
                for (int rr = 0; rr < RG; ++rr)
#pragma unroll
                    for (int c = 0; c < C; ++c)
                        e[rr][c] = dsmem_ld_f2(e_at[c] + static_cast<uint32_t>((r0 + rr) * (NT + NT / 16)) * 8u);
#pragma unroll
                for (int rr = 0; rr < RG; ++rr) {
                    float2 acc = e[rr][0];
#pragma unroll
                    for (int c = 1; c < C; ++c) acc = cadd(acc, quarter_turn(e[rr][c], (rank * c * (4 / C)) & 3));
                    v[r0 + rr] = rank == 0 ? acc : cmul(acc, cmul(xtw_t, xtw_r[r0 + rr]));
                }
            }
        }
        // 4096-point FFT of u, as the one-SM kernel: pass 0 -> P, 1 P -> Q, 2 Q -> registers
        float2* const P = (j & 1) ? xb1 : xb0;
        float2* const Q = (j & 1) ? xb0 : xb1;
        dft16(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) P[fpad(16 * tf + r)] = v[r];
        __syncthreads();                                          // (A)
        {
            const int k = tf & 15;
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = P[fpad(tf + r * NT)];
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw[(r - 1) * 16 + k]);
            dft16(v);
            const int base = (tf >> 4) * 256 + k;
#pragma unroll
            for (int r = 0; r < 16; ++r) Q[fpad(base + r * 16)] = v[r];
        }
        __syncthreads();                                          // (B)
        {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = Q[fpad(tf + r * NT)];
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw[240 + (r - 1) * 256 + tf]);
            dft16(v);                                             // v[r] = Y_rank[k1], k1 = tf + 256 r
        }
#pragma unroll
        for (int r = 0; r < 16; ++r) P[fpad(tf + r * NT)] = v[r];
        cluster_sync();                                           // (S2) every Y_c in its P
        // output bins k = 4096 rank + i, i = tf + 256 r: k2 = tf % C, k1 = k / C
        const uint32_t p_k2 = dsmem_map(P, static_cast<uint32_t>(tf % C));
        const bool bulk = a.full_bulk != 0;
        if (a.full) {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int k1 = (NB / C) * rank + (NT / C) * r + tf / C;
                v[r] = dsmem_ld_f2(p_k2 + static_cast<uint32_t>(fpad(k1)) * 8u);
            }
            if (bulk) {
#pragma unroll
                for (int r = 0; r < 16; ++r) Q[tf + r * NT] = v[r];
                fence_proxy_async_smem();
            } else {
                float2* row = a.full + (a.frame_offset + j) * a.full_ld + rank * NB;
#pragma unroll
                for (int r = 0; r < 16; ++r) row[tf + r * NT] = v[r];
            }
        }
        // this CTA's tones t0 .. t1 - 1
        const int q = static_cast<int>((a.frame_offset + j) & (kToneGroup - 1));
        if (ntc > 0) {
            float2 tv[kTonesPerThread];
            int tb[kTonesPerThread];
#pragma unroll
            for (int k = 0; k < kTonesPerThread; ++k) {
                const int i = tid + k * NT;
                tb[k] = i < t1 - t0 ? sbins[i] : -1;
            }
#pragma unroll
            for (int k = 0; k < kTonesPerThread; ++k)
                if (tb[k] >= 0)
                    tv[k] = dsmem_ld_f2(dsmem_map(P, static_cast<uint32_t>(tb[k] % C)) +
                                        static_cast<uint32_t>(fpad(tb[k] / C)) * 8u);
#pragma unroll
            for (int k = 0; k < kTonesPerThread; ++k)
                if (tb[k] >= 0) tile[(tid + k * NT) * kToneGroup + q] = tv[k];
        } else {
            float2* col = a.tones + a.frame_offset + j;
            for (int t = t0 + tid; t < t1; t += NT) {
                const int bin = __ldg(a.bins + t);
                col[static_cast<int64_t>(t) * a.tones_ld] =
                    dsmem_ld_f2(dsmem_map(P, static_cast<uint32_t>(bin % C)) + static_cast<uint32_t>(fpad(bin / C)) * 8u);
            }
        }
        const bool group_end = ntc > 0 && t1 > t0 && (q == kToneGroup - 1 || j == jb - 1);
        const bool gtma = group_end && a.tones_tma && q == kToneGroup - 1 && j - q >= ja;
        if (gtma) fence_proxy_async_smem();
        __syncthreads();                                          // (C) row piece and tile written
        if (tid == 0) {
            if (a.full && bulk)
                tma_bulk_s2g(a.full + (a.frame_offset + j) * a.full_ld + rank * NB, Q, NB * 8);
            if (gtma) {
                const int32_t x0 = static_cast<int32_t>(a.frame_offset + j - q);
                for (int r0 = 0; r0 < t1 - t0; r0 += kToneBox)
                    tma_store_2d(&tm_tones, x0, t0 + r0, tile + static_cast<size_t>(r0) * kToneGroup);
            }
            bulk_commit();
        }
        if (group_end && !gtma) {
            const int q0 = static_cast<int>(max_i64(0, ja - (j - q)));
            const int nq = q + 1 - q0;
            float2* base = a.tones + a.frame_offset + (j - q);
            for (int it = tid; it < nq * (t1 - t0); it += NT) {
                const int t = it / nq, qq = q0 + (it - t * nq);
                base[static_cast<int64_t>(t0 + t) * a.tones_ld + qq] = tile[t * kToneGroup + qq];
            }
        }
    }
    if (tid == 0) bulk_wait_all();
    umma::fence_before_sync();
    __syncthreads();
    cluster_sync();                                               // no peer reads this CTA's buffers any more
    if (warp == 0) {
        umma::fence_after_sync();
        umma::dealloc(*tmem_holder, 512);
    }
}

// -------------------------------------------------------------- DIRECT
// PRE: the frames' FIR sums come from a.pre (fir_pre_kernel) instead of
// the in-kernel FIR.  Launched with max(N/16, 256) threads; below N = 8192
// four CTAs per SM with the in-kernel FIR (64 registers), two with PRE.
template <int LOG2N, bool PRE>
__global__ void __launch_bounds__(LOG2N >= 14 ? 1024 : (LOG2N == 13 ? 512 : 256),
                                  LOG2N >= 13 ? 1 : (PRE ? 2 : 4))
    pfb_direct_kernel(const PfbArgs a) {
    constexpr int N = 1 << LOG2N;
    constexpr int NT = N / 16;
    constexpr int FSTRIDE = N + N / 16;
    extern __shared__ __align__(1024) unsigned char smem[];
    float2* xbuf = reinterpret_cast<float2*>(smem);
    const int G = blockDim.x / NT;
    const int tid = threadIdx.x;
    const int g = tid / NT, tf = tid % NT;
    const int T = a.T;
    const int64_t n_iter = (a.F + G - 1) / G;
    for (int64_t q = blockIdx.x; q < n_iter; q += gridDim.x) {
        const int64_t j0 = q * G;
        const int64_t j = j0 + g;
        const bool valid = j < a.F;
        float2 v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = make_float2(0.f, 0.f);
        if (PRE && valid) {
            // the frame's FIR sums, computed ahead by fir_pre_kernel (the
            // same FMA chain as the loop below)
            const float2* row = a.pre + j * N + tf;
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = __ldg(row + r * NT);
            // the next frame's rows on their way to L2 (one request per
            // 128-byte line: 16 consecutive points; at N = 16384 it costs a
            // few spilled registers and still measured 9 % faster)
            const int64_t jn = j + static_cast<int64_t>(gridDim.x) * G;
            if (jn < a.F && (tf & 15) == 0) {
                const float2* nrow = a.pre + jn * N + tf;
#pragma unroll
                for (int r = 0; r < 16; ++r) prefetch_l2(nrow + r * NT);
            }
        } else if (!PRE && valid) {
            for (int t = 0; t < T; ++t) {
                const int64_t base = (j + t) * N + tf;
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const float hv = __ldg(a.h + t * N + tf + r * NT);
                    const float2 x = iq_to_f2(vload(a, base + r * NT));
                    v[r].x = fmaf(hv, x.x, v[r].x);
                    v[r].y = fmaf(hv, x.y, v[r].y);
                }
            }
        }
        __syncthreads();   // previous iteration's gather is done with xbuf
        fft_frame<LOG2N, false>(v, xbuf + g * FSTRIDE, tf, a.tw);
        pfb_outputs<LOG2N>(a, v, xbuf, g, tf, j, valid, G, j0);
    }
}

// ------------------------------------------------------------ launcher
namespace {

template <int LOG2N, int T>
size_t ring_smem_bytes(int rs, int tw_count) {
    constexpr int N = 1 << LOG2N;
    constexpr int G = kRingThreads / (N / 16);
    return static_cast<size_t>(rs) * kSB * 4 + static_cast<size_t>(G) * (N + N / 16) * 8 +
           static_cast<size_t>((tw_count + 1) & ~1) * 8 + static_cast<size_t>(rs) * 8;
}

template <int LOG2N, int T>
cudaError_t launch_ring(PfbArgs a, int n_sms, int max_smem, int lookahead, cudaStream_t st) {
    constexpr int N = 1 << LOG2N;
    constexpr int G = kRingThreads / (N / 16);
    constexpr int HB = (T - 1 + G - 1) / G;
    int rs = HB + 1 + ((lookahead >= 1 && lookahead <= 3) ? lookahead : 3);
    while (rs > HB + 2 && ring_smem_bytes<LOG2N, T>(rs, a.tw_count) > static_cast<size_t>(max_smem)) --rs;
    const size_t smem = ring_smem_bytes<LOG2N, T>(rs, a.tw_count);
    if (smem > static_cast<size_t>(max_smem)) return cudaErrorInvalidConfiguration;
    a.ring_sb = rs;
    a.q_lo = (T - 1) / G;
    a.q_hi = (a.F + T - 1 + G - 1) / G;
    const int64_t iters = a.q_hi - a.q_lo;
    const int64_t grid = std::min<int64_t>(iters, n_sms);
    a.iters_per_cta = (iters + grid - 1) / grid;
    const int64_t grid2 = (iters + a.iters_per_cta - 1) / a.iters_per_cta;
    auto k = pfb_ring_kernel<LOG2N, T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<static_cast<unsigned>(grid2), kRingThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int LOG2N>
cudaError_t launch_direct(PfbArgs a, int n_sms, int max_smem, cudaStream_t st) {
    constexpr int N = 1 << LOG2N;
    constexpr int NT = N / 16;
    const int threads = NT >= 256 ? NT : 256;
    const int G = threads / NT;
    const size_t smem = static_cast<size_t>(G) * (N + N / 16) * 8;
    if (smem > static_cast<size_t>(max_smem)) return cudaErrorInvalidConfiguration;
    const int64_t n_iter = (a.F + G - 1) / G;
    int per_sm = 1;
    // pre-sum instances only for the shapes that take them (pfb_pre_rows)
    constexpr bool kPre = (LOG2N >= 8 && LOG2N <= 11) || LOG2N == 13 || LOG2N == 14;
    if (a.pre && !kPre) return cudaErrorInvalidValue;
    auto k = a.pre ? pfb_direct_kernel<LOG2N, kPre> : pfb_direct_kernel<LOG2N, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(n_iter, static_cast<int64_t>(n_sms) * std::max(per_sm, 1)));
    k<<<static_cast<unsigned>(grid), threads, smem, st>>>(a);
    return cudaGetLastError();
}

// FIR sums of the first T (<= TMAX) taps of every frame of the stream view
// [carry | buffer] (N channels):
//   pre[j][p] = sum_{t<T} h[t N + p] x[(j + t) N + p],
// FMAs in tap order from zero, the order of the fused kernels' FIRs, which
// continue these sums (the 16-tap N = 4096 form: taps 0..7 here, 8..15 in
// the TMEM kernel) or take them whole (the direct kernel).  A thread takes
// P points (kPreThreads apart) of G consecutive frames and loads and
// converts each of their G + T - 1 input blocks once; the frame
// groups of a point range are consecutive CTAs, so the blocks two groups
// share and the range's taps come from DRAM once.
constexpr int kPreThreads = 256;
template <int TMAX, int P, int G, int LOG2N, bool EXACT>
__global__ void __launch_bounds__(kPreThreads) fir_pre_kernel(const PfbArgs a, int T_arg, float2* __restrict__ pre) {
    constexpr int N = 1 << LOG2N, R = G + TMAX - 1;
    const int T = EXACT ? TMAX : T_arg;              // EXACT: T == TMAX, known at compile time
    const int64_t f0 = static_cast<int64_t>(blockIdx.x) * G;
    const int gn = static_cast<int>(min_i64(a.F - f0, G));
    const int qb = static_cast<int>(blockIdx.y) * (kPreThreads * P) + static_cast<int>(threadIdx.x);
    float hv[TMAX][P];
#pragma unroll
    for (int t = 0; t < TMAX; ++t)
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const int q = qb + k * kPreThreads;
            hv[t][k] = (t < T && q < N) ? __ldg(a.h + t * N + q) : 0.f;
        }
    const int64_t base = f0 * N + qb;
    uint32_t w[R][P];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < P; ++k)
            w[r][k] = (r < gn + T - 1 && qb + k * kPreThreads < N)
                          ? vload(a, base + static_cast<int64_t>(r) * N + k * kPreThreads) : 0u;
    float ar[G][P], ai[G][P];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int k = 0; k < P; ++k) ar[g][k] = ai[g][k] = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const float2 x = iq_to_f2(w[r][k]);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int t = r - g;
                if (t < 0 || t >= TMAX || t >= T) continue;
                ar[g][k] = fmaf(hv[t][k], x.x, ar[g][k]);
                ai[g][k] = fmaf(hv[t][k], x.y, ai[g][k]);
            }
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (g >= gn) break;
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const int q = qb + k * kPreThreads;
            if (q < N) pre[(f0 + g) * N + q] = make_float2(ar[g][k], ai[g][k]);
        }
    }
}

// The pre-sum rows of the first T taps of a.F frames (2^lg channels) into
// pre: instances for the shapes that take them (rfr::pfb_pre_rows).
template <int TMAX, int P, int G, int LOG2N>
cudaError_t launch_pre_n(const PfbArgs& a, int T, float2* pre, cudaStream_t st) {
    const dim3 g(static_cast<unsigned>((a.F + G - 1) / G),
                 static_cast<unsigned>(((1 << LOG2N) + kPreThreads * P - 1) / (kPreThreads * P)));
    if (T == TMAX)
        fir_pre_kernel<TMAX, P, G, LOG2N, true><<<g, kPreThreads, 0, st>>>(a, T, pre);
    else
        fir_pre_kernel<TMAX, P, G, LOG2N, false><<<g, kPreThreads, 0, st>>>(a, T, pre);
    return cudaGetLastError();
}
// Eight frames per thread (each block reloaded (8 + T - 1) / 8 times per
// frame instead of (4 + T - 1) / 4) and few points (fewer registers, more
// warps per SM) measured 9-25 % faster than four frames of four or two
// points at N = 16384.
cudaError_t launch_pre(const PfbArgs& a, int lg, int T, float2* pre, cudaStream_t st) {
    if (T < 1 || T > 16) return cudaErrorInvalidValue;
    if (T <= 8) {
        switch (lg) {
        case 12: return launch_pre_n<8, 2, 8, 12>(a, T, pre, st);
        case 13: return launch_pre_n<8, 2, 8, 13>(a, T, pre, st);
        case 14: return launch_pre_n<8, 2, 8, 14>(a, T, pre, st);
        default: return cudaErrorInvalidValue;
        }
    }
    // more taps: one point and eight frames per thread
    switch (lg) {
    case 8: return launch_pre_n<16, 1, 8, 8>(a, T, pre, st);
    case 9: return launch_pre_n<16, 1, 8, 9>(a, T, pre, st);
    case 10: return launch_pre_n<16, 1, 8, 10>(a, T, pre, st);
    case 11: return launch_pre_n<16, 1, 8, 11>(a, T, pre, st);
    case 13: return launch_pre_n<16, 1, 8, 13>(a, T, pre, st);
    case 14: return launch_pre_n<16, 1, 8, 14>(a, T, pre, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int T, bool PRE = false>
cudaError_t launch_tmem(PfbArgs a, int n_sms, int max_smem, cudaStream_t st) {
    a.nb_smem = (a.n_tones > 0 && a.n_tones <= kTonesPerThread * kRingThreads &&
                 tmem_layout(a.tw_count, a.n_tones).total <= static_cast<size_t>(max_smem))
                    ? a.n_tones : 0;
    const size_t smem = tmem_layout(a.tw_count, a.nb_smem).total;
    if (smem > static_cast<size_t>(max_smem)) return cudaErrorInvalidConfiguration;
    // whole tone groups per CTA (of output frames, see the kernel)
    const int64_t shift = a.frame_offset & (kToneGroup - 1);
    const int64_t grid = std::min<int64_t>(a.F, n_sms);
    a.iters_per_cta = ((a.F + shift + grid - 1) / grid + kToneGroup - 1) / kToneGroup * kToneGroup;
    const int64_t grid2 = (a.F + shift + a.iters_per_cta - 1) / a.iters_per_cta;
    a.full_bulk = (a.full != nullptr && (reinterpret_cast<uintptr_t>(a.full) % 16) == 0 &&
                   (a.full_ld % 2) == 0) ? 1 : 0;
    // tone rows as a 2-D tensor of 8-byte elements [n_tones][frame_offset + F]
    // (row pitch tones_ld * 8 bytes, a multiple of 16); box kToneGroup x kToneBox
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    a.tones_tma = 0;
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tmap_encode_tiled_fn());
    if (a.nb_smem > 0 && enc && (reinterpret_cast<uintptr_t>(a.tones) % 16) == 0 && (a.tones_ld % 2) == 0 &&
        a.frame_offset + a.F < (int64_t(1) << 31)) {
        cuuint64_t dims[2] = {static_cast<cuuint64_t>(a.frame_offset + a.F), static_cast<cuuint64_t>(a.n_tones)};
        cuuint64_t strides[1] = {static_cast<cuuint64_t>(a.tones_ld) * 8};
        cuuint32_t box[2] = {kToneGroup, kToneBox};
        cuuint32_t estr[2] = {1, 1};
        if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, a.tones, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
            a.tones_tma = 1;
    }
    auto k = pfb_tmem_kernel<T, PRE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<static_cast<unsigned>(grid2), kRingThreads, smem, st>>>(a, tm);
    return cudaGetLastError();
}

cudaError_t launch_tmem_sym(PfbArgs a, int n_sms, int max_smem, cudaStream_t st) {
    a.nb_smem = (a.n_tones > 0 && a.n_tones <= kTonesPerThread * kRingThreads &&
                 sym_layout(a.n_tones).total <= static_cast<size_t>(max_smem))
                    ? a.n_tones : 0;
    const size_t smem = sym_layout(a.nb_smem).total;
    if (smem > static_cast<size_t>(max_smem)) return cudaErrorInvalidConfiguration;
    const int64_t shift = a.frame_offset & (kToneGroup - 1);
    const int64_t grid = std::min<int64_t>(a.F, n_sms);
    a.iters_per_cta = ((a.F + shift + grid - 1) / grid + kToneGroup - 1) / kToneGroup * kToneGroup;
    const int64_t grid2 = (a.F + shift + a.iters_per_cta - 1) / a.iters_per_cta;
    a.full_bulk = (a.full != nullptr && (reinterpret_cast<uintptr_t>(a.full) % 16) == 0 &&
                   (a.full_ld % 2) == 0) ? 1 : 0;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    a.tones_tma = 0;
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tmap_encode_tiled_fn());
    if (a.nb_smem > 0 && enc && a.tone_cs == 1 && (reinterpret_cast<uintptr_t>(a.tones) % 16) == 0 &&
        (a.tones_ld % 2) == 0 && a.frame_offset + a.F < (int64_t(1) << 31)) {
        cuuint64_t dims[2] = {static_cast<cuuint64_t>(a.frame_offset + a.F), static_cast<cuuint64_t>(a.n_tones)};
        cuuint64_t strides[1] = {static_cast<cuuint64_t>(a.tones_ld) * 8};
        cuuint32_t box[2] = {kToneGroup, kToneBox};
        cuuint32_t estr[2] = {1, 1};
        if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, a.tones, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
            a.tones_tma = 1;
    }
    const bool phase = a.tone_cs != 1 || a.rot != 0;
    auto k = phase ? pfb_tmem_sym_kernel<true> : pfb_tmem_sym_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<static_cast<unsigned>(grid2), kRingThreads, smem, st>>>(a, tm);
    return cudaGetLastError();
}

template <int C, int T>
cudaError_t launch_cluster(PfbArgs a, int n_sms, int max_smem, cudaStream_t st) {
    // tone rows per CTA: whole 256-row boxes, so no CTA's tone stores reach
    // another CTA's rows
    int ntc = 0;
    if (a.n_tones > 0) {
        ntc = ((a.n_tones + C - 1) / C + kToneBox - 1) / kToneBox * kToneBox;
        if (ntc > kClusterTonesPerCta || cluster_layout(a.tw_count, ntc).total > static_cast<size_t>(max_smem)) ntc = 0;
    }
    a.nb_smem = ntc;
    const size_t smem = cluster_layout(a.tw_count, ntc).total;
    if (smem > static_cast<size_t>(max_smem)) return cudaErrorInvalidConfiguration;
    auto k = pfb_cluster_kernel<C, T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kRingThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static int max_clusters[2][2] = {{0, 0}, {0, 0}};             // [C == 4][T == 8], queried once
    int& mc = max_clusters[C == 4 ? 1 : 0][T == 8 ? 1 : 0];
    if (mc <= 0) {
        cfg.gridDim = dim3(static_cast<unsigned>(C * (n_sms / C)), 1, 1);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = n_sms / C;
        }
        mc = n;
    }
    // whole tone groups of output frames per cluster, as the one-SM kernel
    const int64_t shift = a.frame_offset & (kToneGroup - 1);
    const int64_t ncl = std::max<int64_t>(1, std::min<int64_t>(a.F, mc));
    a.iters_per_cta = ((a.F + shift + ncl - 1) / ncl + kToneGroup - 1) / kToneGroup * kToneGroup;
    const int64_t ncl2 = (a.F + shift + a.iters_per_cta - 1) / a.iters_per_cta;
    a.full_bulk = (a.full != nullptr && (reinterpret_cast<uintptr_t>(a.full) % 16) == 0 &&
                   (a.full_ld % 2) == 0) ? 1 : 0;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    a.tones_tma = 0;
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tmap_encode_tiled_fn());
    if (ntc > 0 && enc && (reinterpret_cast<uintptr_t>(a.tones) % 16) == 0 && (a.tones_ld % 2) == 0 &&
        a.frame_offset + a.F < (int64_t(1) << 31)) {
        cuuint64_t dims[2] = {static_cast<cuuint64_t>(a.frame_offset + a.F), static_cast<cuuint64_t>(a.n_tones)};
        cuuint64_t strides[1] = {static_cast<cuuint64_t>(a.tones_ld) * 8};
        cuuint32_t box[2] = {kToneGroup, kToneBox};
        cuuint32_t estr[2] = {1, 1};
        if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, a.tones, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
            a.tones_tma = 1;
    }
    cfg.gridDim = dim3(static_cast<unsigned>(C * ncl2), 1, 1);
    e = cudaLaunchKernelEx(&cfg, k, a, tm);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int LOG2N>
cudaError_t dispatch_ring_T(PfbArgs a, int tk, int n_sms, int max_smem, int la, cudaStream_t st) {
    switch (tk) {
    case 4: return launch_ring<LOG2N, 4>(a, n_sms, max_smem, la, st);
    case 8: return launch_ring<LOG2N, 8>(a, n_sms, max_smem, la, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool pfb_uses_ring(int log2n, int taps) { return log2n >= 4 && log2n <= 12 && taps <= 8; }
int pfb_cluster_size(int log2n, int taps) { return (log2n == 13 || log2n == 14) && taps <= 8 ? 1 << (log2n - 12) : 0; }
bool pfb_split16(int log2n, int taps) { return log2n == 12 && taps == 16; }
// Where the direct kernel takes its FIR from a pre-sum pass (measured, 2^28
// samples, full + tones): N = 8192 at every T (T = 8: 3.14 -> 1.81 ms),
// N = 16384 from T = 8 on (2.73 -> 1.85 ms; T = 4 1.87 -> 2.14 ms, so not
// there), N = 256 .. 2048 with T > 8 (T = 16: N = 1024 5.39 -> 3.15 ms,
// N = 256 with 64 tones 4.39 -> 1.61 ms).  Smaller N, or T <= 8 below
// N = 4096, run on the shared-memory ring kernel.
bool pfb_pre_rows(int log2n, int taps) {
    if (pfb_split16(log2n, taps)) return true;
    if (log2n == 13) return true;
    if (log2n == 14) return taps > 4;
    return log2n >= 8 && log2n <= 11 && taps > 8;
}
int pfb_kernel_taps(int log2n, int taps) {
    if (pfb_uses_ring(log2n, taps) || pfb_cluster_size(log2n, taps) > 0) return taps <= 4 ? 4 : 8;
    if (log2n == 12 && taps > 8 && taps <= 16) return 16;     // first-half pass + seeded TMEM kernel (pfb_launch)
    return taps;
}

cudaError_t pfb_launch(const PfbLaunch& L, cudaStream_t st) {
    PfbArgs a{};
    a.carry = reinterpret_cast<const uint32_t*>(L.carry);
    a.cl = L.cl;
    a.buf = reinterpret_cast<const uint32_t*>(L.buf);
    a.n = L.n;
    a.F = L.F;
    a.h = L.h;
    a.tw = reinterpret_cast<const float2*>(L.tw);
    a.tw_count = L.tw_count;
    a.T = L.taps_kernel;
    a.bins = L.bins;
    a.n_tones = L.n_tones;
    a.full = reinterpret_cast<float2*>(L.full);
    a.full_ld = L.full_ld;
    a.tones = reinterpret_cast<float2*>(L.tones);
    a.tones_ld = L.tones_ld;
    a.frame_offset = L.frame_offset;
    a.status = L.status;
    a.tone_cs = L.tone_cs > 0 ? L.tone_cs : 1;
    a.rot = L.rot & 3;
    if (a.F <= 0) return cudaSuccess;
    const bool aligned = (reinterpret_cast<uintptr_t>(L.buf) % 16 == 0) && (L.cl % 4 == 0) &&
                         (reinterpret_cast<uintptr_t>(L.carry) % 16 == 0);
    a.use_tma = aligned ? 1 : 0;
    const int lg = L.log2n;
    if (L.cluster && pfb_cluster_size(lg, L.taps_kernel) > 0) {
        // N = 8192 or 16384, T <= 8 on the cluster kernel (when the plan
        // chose it), aligned or not
        if (a.tone_cs != 1 || a.rot != 0 || !L.tw_cl) return cudaErrorInvalidValue;
        a.tw = reinterpret_cast<const float2*>(L.tw_cl);
        a.tw_count = L.tw_cl_count;
        if (lg == 13) return L.taps_kernel == 4 ? launch_cluster<2, 4>(a, L.n_sms, L.max_smem, st)
                                                : launch_cluster<2, 8>(a, L.n_sms, L.max_smem, st);
        return L.taps_kernel == 4 ? launch_cluster<4, 4>(a, L.n_sms, L.max_smem, st)
                                  : launch_cluster<4, 8>(a, L.n_sms, L.max_smem, st);
    }
    if (pfb_split16(lg, L.taps_kernel)) {
        // N = 4096, T = 16 (9 .. 16 taps, zero-padded at the oldest end):
        // the FIR of taps 0..7 over the window's first 8 blocks by
        // fir_pre_kernel into L.pre, then the TMEM kernel over the view 8N
        // samples on with taps 8..15, its FIR sums starting from those rows
        // (the same FMA chain as one 16-tap FIR).  The caller passes a
        // 16-byte aligned view and L.pre for at least F frames.
        if (a.tone_cs != 1 || a.rot != 0 || !a.use_tma || !L.pre || L.pre_cap < a.F) return cudaErrorInvalidValue;
        constexpr int64_t half = int64_t(8) * 4096;
        PfbArgs a1 = a;
        a1.T = 8;
        cudaError_t e = launch_pre(a1, 12, 8, static_cast<float2*>(L.pre), st);
        if (e != cudaSuccess) return e;
        PfbArgs a2 = a1;
        a2.h = a.h + half;
        if (a.cl >= half) {
            a2.carry = a.carry + half;
            a2.cl = a.cl - half;
        } else {
            a2.carry = a.carry;
            a2.cl = 0;
            a2.buf = a.buf + (half - a.cl);
            a2.n = a.n - (half - a.cl);
        }
        a2.pre = static_cast<const float2*>(L.pre);
        return launch_tmem<8, true>(a2, L.n_sms, L.max_smem, st);
    }
    if (a.tone_cs != 1 || a.rot != 0) {
        // phase passes of an oversampled plan: only the symmetric-tap kernel has them
        if (lg != 12 || !a.use_tma || L.taps_kernel != 8 || !L.sym_taps) return cudaErrorInvalidValue;
        return launch_tmem_sym(a, L.n_sms, L.max_smem, st);
    }
    if (lg == 12 && a.use_tma && L.variant != 1) {
        if (L.taps_kernel == 8 && L.sym_taps && L.variant != 2) return launch_tmem_sym(a, L.n_sms, L.max_smem, st);
        if (L.taps_kernel == 4) return launch_tmem<4>(a, L.n_sms, L.max_smem, st);
        if (L.taps_kernel == 8) return launch_tmem<8>(a, L.n_sms, L.max_smem, st);
    }
    if (pfb_uses_ring(lg, L.taps_kernel)) {
        switch (lg) {
        case 4: return dispatch_ring_T<4>(a, L.taps_kernel, L.n_sms, L.max_smem, L.lookahead, st);
        case 5: return dispatch_ring_T<5>(a, L.taps_kernel, L.n_sms, L.max_smem, L.lookahead, st);
        case 6: return dispatch_ring_T<6>(a, L.taps_kernel, L.n_sms, L.max_smem, L.lookahead, st);
        case 7: return dispatch_ring_T<7>(a, L.taps_kernel, L.n_sms, L.max_smem, L.lookahead, st);
        case 8: return dispatch_ring_T<8>(a, L.taps_kernel, L.n_sms, L.max_smem, L.lookahead, st);
        case 9: return dispatch_ring_T<9>(a, L.taps_kernel, L.n_sms, L.max_smem, L.lookahead, st);
        case 10: return dispatch_ring_T<10>(a, L.taps_kernel, L.n_sms, L.max_smem, L.lookahead, st);
        case 11: return dispatch_ring_T<11>(a, L.taps_kernel, L.n_sms, L.max_smem, L.lookahead, st);
        case 12: return dispatch_ring_T<12>(a, L.taps_kernel, L.n_sms, L.max_smem, L.lookahead, st);
        default: return cudaErrorInvalidValue;
        }
    }
    if (L.pre) {
        // the FIR of all taps ahead, as its own DRAM-streaming pass (the
        // direct kernel would re-read every tap and sample T times through L2)
        if (L.pre_cap < a.F) return cudaErrorInvalidValue;
        cudaError_t e = launch_pre(a, lg, L.taps_kernel, static_cast<float2*>(L.pre), st);
        if (e != cudaSuccess) return e;
        a.pre = static_cast<const float2*>(L.pre);
    }
    switch (lg) {
    case 4: return launch_direct<4>(a, L.n_sms, L.max_smem, st);
    case 5: return launch_direct<5>(a, L.n_sms, L.max_smem, st);
    case 6: return launch_direct<6>(a, L.n_sms, L.max_smem, st);
    case 7: return launch_direct<7>(a, L.n_sms, L.max_smem, st);
    case 8: return launch_direct<8>(a, L.n_sms, L.max_smem, st);
    case 9: return launch_direct<9>(a, L.n_sms, L.max_smem, st);
    case 10: return launch_direct<10>(a, L.n_sms, L.max_smem, st);
    case 11: return launch_direct<11>(a, L.n_sms, L.max_smem, st);
    case 12: return launch_direct<12>(a, L.n_sms, L.max_smem, st);
    case 13: return launch_direct<13>(a, L.n_sms, L.max_smem, st);
    case 14: return launch_direct<14>(a, L.n_sms, L.max_smem, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rfr
