// demod.cu -- direct multi-tone demodulation (Sec. III.B of arXiv:1812.02200)
// as the dense contraction it is, on the tcgen05 tensor cores.
//
// Definition (per tone t with NCO word w_t, frame k, b_k = first sample of
// the frame, taps h[0..L)):
//   out[t][k] = sum_n h[n] x[b_k+n] exp(-i*phi_t(b_k+n)),  phi_t(m) = 2*pi*(w_t*m mod 2^64)/2^64.
// Because w_t*(b+n) = w_t*b + w_t*n (mod 2^64) exactly,
//   out[t][k] = exp(-i*phi_t(b_k)) * sum_n x[b_k+n] * C_t[n],   C_t[n] = h[n] exp(-i*phi_t(n)),
// i.e. a GEMM of the Toeplitz matrix A[k][n] = x[b_k+n] (row stride D) with
// the modulated taps C (plan constant), followed by a per-(t,k) rotation.
//
// Precision.  x is a 14-bit integer: x = xh + xl with xh = fp16(x) and
// xl = x - xh, both exact in FP16.  C (scaled by 2^e so max|C| is in
// [2^14, 2^15)) is split into ch = fp16(C) and cl = fp16(C - ch).  The MMAs
// accumulate xh*ch + xh*cl + xl*ch (the dropped xl*cl is ~2^-22 relative) in
// FP32.  To keep the tensor cores' internal accumulation error small, each
// TMEM accumulator collects only a short chunk of K and the epilogue warps add
// the chunks into FP32 register sums (the accumulator is double-buffered, so
// the MMAs of the next chunk overlap the drain of the previous one).
//
// Real embedding: K' = 2L (re, im of x interleaved), N' = 2*tones with
//   B'[2t][2n] = Re C, B'[2t][2n+1] = -Im C, B'[2t+1][2n] = Im C, B'[2t+1][2n+1] = Re C
// so column 2t of the product is Re(x.C_t) and column 2t+1 is Im(x.C_t).
//
// Kernels:
//   build_taps  (plan time) FP64 modulated taps -> FP16 hi/lo, K-major B'.
//   rot         (per push)  FP64 rotation anchors exp(-i*phi_t(b)) at every
//                           128-frame tile start and steps exp(-i*w_t*D*j).
//   presplit    (per push)  int16 IQ of [carry | buffer] -> FP16 hi/lo rows of D
//                           samples (the Toeplitz view's 2-D tensor).
//   gemm        (per push)  TMA -> smem (128B swizzle) -> tcgen05.mma -> TMEM
//                           -> register sums -> rotation -> [tone][frame] out.
//   *3 variants             the Gauss three-product form (see below), a plan
//                           option (rfr_plan_set_demod_products).
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "dev_common.cuh"
#include "rfr_internal.h"
#include "umma.cuh"

namespace rfr {

// the CUDA driver API's cuTensorMapEncodeTiled, looked up once (nullptr if absent)
void* tmap_encode_tiled_fn() {
    static void* fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = p;
    });
    return fn;
}

namespace {

constexpr int BM = kDemodBM, BN = kDemodBN, BK = kDemodBK;
constexpr int STAGES = 2;
constexpr uint32_t A_BYTES = BM * BK * 2;
constexpr uint32_t B_BYTES = BN * BK * 2;
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int EPI_WARPS = 8;
constexpr int GEMM_THREADS = (EPI_WARPS + 2) * 32;
constexpr uint32_t TMEM_COLS = 512;       // two 256-column FP32 accumulators
constexpr size_t GEMM_SMEM = 1024 + STAGES * STAGE_BYTES + 256;

__device__ __forceinline__ float2 expmi_u64(uint64_t phase) {
    // exp(-i * 2*pi*phase/2^64) in FP64, rounded to FP32
    const double xs = static_cast<double>(static_cast<int64_t>(phase)) * 0x1p-63;   // in [-1, 1)
    double s, c;
    sincospi(xs, &s, &c);
    return make_float2(static_cast<float>(c), static_cast<float>(-s));
}

__device__ __forceinline__ void split_store(__half* hi, __half* lo, size_t i, double v) {
    const __half h = __double2half(v);
    hi[i] = h;
    lo[i] = __double2half(v - static_cast<double>(__half2float(h)));
}

__global__ void build_taps_kernel(const double* __restrict__ h, const uint64_t* __restrict__ words,
                                  int n_tones, int ntp, int L, int Lpad, double scale,
                                  __half* __restrict__ bh, __half* __restrict__ bl) {
    const int64_t total = static_cast<int64_t>(ntp) * Lpad;
    const size_t ldk = static_cast<size_t>(2) * Lpad;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int t = static_cast<int>(idx / Lpad);
        const int n = static_cast<int>(idx - static_cast<int64_t>(t) * Lpad);
        double cr = 0.0, ci = 0.0;
        if (t < n_tones && n < L) {
            const uint64_t ph = words[t] * static_cast<uint64_t>(n);
            const double xs = static_cast<double>(static_cast<int64_t>(ph)) * 0x1p-63;
            double s, c;
            sincospi(xs, &s, &c);
            const double a = h[n] * scale;
            cr = a * c;      // C = h * exp(-i*theta) = h*(cos - i sin)
            ci = -a * s;
        }
        const size_t r0 = static_cast<size_t>(2 * t) * ldk, r1 = r0 + ldk;
        split_store(bh, bl, r0 + 2 * n, cr);
        split_store(bh, bl, r0 + 2 * n + 1, -ci);
        split_store(bh, bl, r1 + 2 * n, ci);
        split_store(bh, bl, r1 + 2 * n + 1, cr);
    }
}

// Rotation factors on ABSOLUTE frame indices K = 128*A + i (so a stream split
// into pushes rotates every frame by the same FP32 factors):
//   anchors[a] = exp(-i*phi_t(b(128*(A0 + a)))),  steps[t][i] = exp(-i*w_t*D*i),
// with b(K) = (K+1)*D - L the first sample of frame K and A0 = F0/128.
__global__ void rot_kernel(const uint64_t* __restrict__ words, int n_tones, int ntp, int64_t A0, int L,
                           int D, int n_anch, float2* __restrict__ anchors, float2* __restrict__ steps) {
    const int64_t na = static_cast<int64_t>(n_anch) * ntp;
    const int64_t total = na + static_cast<int64_t>(ntp) * BM;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (idx < na) {
            const int a = static_cast<int>(idx / ntp);
            const int t = static_cast<int>(idx - static_cast<int64_t>(a) * ntp);
            float2 r = make_float2(0.f, 0.f);
            if (t < n_tones) {
                const int64_t K = (A0 + a) * BM;
                const int64_t b = (K + 1) * D - L;
                r = expmi_u64(words[t] * static_cast<uint64_t>(b));
            }
            anchors[idx] = r;
        } else {
            const int64_t j = idx - na;
            const int t = static_cast<int>(j / BM);
            const int i = static_cast<int>(j - static_cast<int64_t>(t) * BM);
            float2 r = make_float2(0.f, 0.f);
            if (t < n_tones) r = expmi_u64(words[t] * static_cast<uint64_t>(static_cast<int64_t>(i) * D));
            steps[j] = r;
        }
    }
}

// Sample s of the virtual stream [carry | buffer] -> FP16 hi/lo pairs.
__global__ void presplit_kernel(const uint32_t* __restrict__ carry, int64_t cl,
                                const uint32_t* __restrict__ buf, int64_t lv, int64_t total,
                                __half2* __restrict__ hi, __half2* __restrict__ lo) {
    for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < total;
         s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint32_t w = 0;
        if (s < lv) w = s < cl ? carry[s] : buf[s - cl];
        const float2 f = iq_to_f2(w);
        const __half hr = __float2half_rn(f.x), hq = __float2half_rn(f.y);
        hi[s] = __halves2half2(hr, hq);
        lo[s] = __halves2half2(__float2half_rn(f.x - __half2float(hr)),
                               __float2half_rn(f.y - __half2float(hq)));
    }
}

struct GemmArgs {
    int raster;           // tile order: groups of `raster` M tiles sweep all N tiles
    int64_t F;
    int64_t F0;           // frames of the stream before this push
    int n_tones, ntp, KB, kchunk, two_d, n_mt, n_nt;
    const float2* anchors;
    const float2* steps;
    float inv_scale;
    float2* out;
    int64_t ld, fo;
    int* status;
};

// Tile index -> (M tile, N tile): groups of g.raster M tiles are swept
// N-tile-major, so concurrently running CTAs share the same tap slices in L2.
__device__ __forceinline__ void tile_coords_of(int raster, int n_mt, int n_nt, int tile, int& mt, int& nt) {
    const int r = raster > 1 ? raster : 1;
    if (r == 1) {
        mt = tile / n_nt;
        nt = tile % n_nt;
        return;
    }
    const int per_group = r * n_nt;
    const int grp = tile / per_group, in = tile % per_group;
    const int m_base = grp * r;
    const int rows = min(r, n_mt - m_base);
    nt = in / rows;
    mt = m_base + in % rows;
}
__device__ __forceinline__ void tile_coords(const GemmArgs& g, int tile, int& mt, int& nt) {
    tile_coords_of(g.raster, g.n_mt, g.n_nt, tile, mt, nt);
}

__global__ void __launch_bounds__(GEMM_THREADS, 1)
demod_gemm_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                  const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                  const GemmArgs g) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tempty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EPI_WARPS * 32);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == EPI_WARPS + 1) {
        umma::alloc(tmem_holder, TMEM_COLS);
        umma::relinquish();
    }
    if (warp == EPI_WARPS && lane == 0) {
        tma_prefetch_desc(&tmAh);
        tma_prefetch_desc(&tmAl);
        tma_prefetch_desc(&tmBh);
        tma_prefetch_desc(&tmBl);
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    const int n_tiles = g.n_mt * g.n_nt;
    constexpr uint32_t IDESC = umma::idesc_f16_f32(BM, BN);

    if (warp == EPI_WARPS) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            for (int tile = blockIdx.x; tile < n_tiles && !*abort_flag; tile += gridDim.x) {
                int tm, tn;
                tile_coords(g, tile, tm, tn);
                const int m0 = tm * BM, n0 = tn * BN;
                for (int kb = 0; kb < g.KB; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1, g.status)) { *abort_flag = 1; break; }
                    unsigned char* st = smem + s * STAGE_BYTES;
                    mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                    const int kh = kb * BK;
                    const int c0 = kh % g.two_d, c1 = m0 + kh / g.two_d;
                    tma_load_2d(st, &tmAh, c0, c1, &full[s]);
                    tma_load_2d(st + A_BYTES, &tmAl, c0, c1, &full[s]);
                    tma_load_2d(st + 2 * A_BYTES, &tmBh, kh, n0, &full[s]);
                    tma_load_2d(st + 2 * A_BYTES + B_BYTES, &tmBl, kh, n0, &full[s]);
                }
            }
            // wait for the copies still in flight before leaving
            for (uint32_t k = 0; k < STAGES && it > 0; ++k) {
                const uint32_t j = it - 1 - k;
                if (static_cast<int32_t>(j) < 0) break;
                // the last STAGES fills: their full barriers complete on arrival
                mbar_wait(&full[j % STAGES], (j / STAGES) & 1, g.status);
            }
        }
    } else if (warp == EPI_WARPS + 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t it = 0, cc = 0;
            for (int tile = blockIdx.x; tile < n_tiles && !*abort_flag; tile += gridDim.x) {
                for (int kb0 = 0; kb0 < g.KB && !*abort_flag; kb0 += g.kchunk, ++cc) {
                    const uint32_t ab = cc & 1, aph = (cc >> 1) & 1;
                    if (!mbar_wait(&tempty[ab], aph ^ 1, g.status)) { *abort_flag = 1; break; }
                    umma::fence_after_sync();
                    const uint32_t d_tmem = tmem + ab * BN;
                    const int kb1 = min(kb0 + g.kchunk, g.KB);
                    for (int kb = kb0; kb < kb1; ++kb, ++it) {
                        const int s = it % STAGES;
                        const uint32_t ph = (it / STAGES) & 1;
                        if (!mbar_wait(&full[s], ph, g.status)) { *abort_flag = 1; break; }
                        umma::fence_after_sync();
                        const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                        const uint32_t ah = sa, al = sa + A_BYTES;
                        const uint32_t bh = sa + 2 * A_BYTES, bl = bh + B_BYTES;
#pragma unroll
                        for (int k = 0; k < BK / 16; ++k) {
                            const uint32_t off = k * 32;   // 16 fp16 of K = 32 bytes
                            const uint32_t acc = (kb > kb0 || k > 0) ? 1u : 0u;
                            umma::mma_f16(d_tmem, umma::desc_k_sw128(ah + off), umma::desc_k_sw128(bh + off), IDESC, acc);
                            umma::mma_f16(d_tmem, umma::desc_k_sw128(ah + off), umma::desc_k_sw128(bl + off), IDESC, 1u);
                            umma::mma_f16(d_tmem, umma::desc_k_sw128(al + off), umma::desc_k_sw128(bh + off), IDESC, 1u);
                        }
                        umma::commit(&empty[s]);
                    }
                    umma::commit(&tfull[ab]);
                }
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue (8 warps)
        const int q = warp & 3, half_sel = warp >> 2;
        const int row = q * 32 + lane;
        uint32_t cc = 0;
        for (int tile = blockIdx.x; tile < n_tiles && !*abort_flag; tile += gridDim.x) {
            int mt, tn;
            tile_coords(g, tile, mt, tn);
            const int m0 = mt * BM, n0 = tn * BN;
            float sums[128];
#pragma unroll
            for (int i = 0; i < 128; ++i) sums[i] = 0.f;
            bool ok = true;
            for (int kb0 = 0; kb0 < g.KB; kb0 += g.kchunk, ++cc) {
                const uint32_t ab = cc & 1, aph = (cc >> 1) & 1;
                if (!mbar_wait(&tfull[ab], aph, g.status)) { *abort_flag = 1; ok = false; break; }
                umma::fence_after_sync();
                const uint32_t base = tmem + (static_cast<uint32_t>(q * 32) << 16) + ab * BN + half_sel * 128;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint32_t r[32];
                    umma::ld_32x32b_x32(base + j * 32, r);
                    umma::wait_ld();
#pragma unroll
                    for (int i = 0; i < 32; ++i) sums[j * 32 + i] += __uint_as_float(r[i]);
                }
                umma::fence_before_sync();
                mbar_arrive(&tempty[ab]);
            }
            if (!ok) break;
            const int64_t k = static_cast<int64_t>(m0) + row;
            if (k < g.F) {
                const int tb = n0 / 2 + half_sel * 64;
                const int64_t K = g.F0 + k;                       // absolute frame
                const int64_t arow = K / BM - g.F0 / BM;          // anchor row of this push
                const int si = static_cast<int>(K % BM);
#pragma unroll
                for (int tl = 0; tl < 64; ++tl) {
                    const int t = tb + tl;
                    if (t < g.n_tones) {
                        const float2 an = __ldg(g.anchors + arow * g.ntp + t);
                        const float2 sp = __ldg(g.steps + static_cast<int64_t>(t) * BM + si);
                        const float2 rot = cmul(an, sp);
                        const float2 acc = make_float2(sums[2 * tl] * g.inv_scale, sums[2 * tl + 1] * g.inv_scale);
                        g.out[static_cast<int64_t>(t) * g.ld + g.fo + k] = cmul(acc, rot);
                    }
                }
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == EPI_WARPS + 1) {
        umma::fence_after_sync();
        umma::dealloc(tmem, TMEM_COLS);
    }
}

// ---------------------------------------------- Gauss three-product form
//
// With x = xr + i xi and C = cr + i ci, the three real contractions
//   P1 = sum ((xr + xi)/2) cr,   P2 = sum xr (ci - cr),   P3 = sum xi (cr + ci)
// give Re(x.C) = 2 P1 - P3 and Im(x.C) = 2 P1 + P2: three real products per
// complex multiply-add instead of the four of the real embedding.  Each A
// plane ((xr+xi)/2, xr, xi) and B plane (cr, ci-cr, cr+ci) is split into FP16
// hi/lo as above ((xr+xi)/2 has at most 17 significant bits, exact as hi+lo);
// each product again takes the three MMAs hi.hi + hi.lo + lo.hi.
//
// Tile: 128 frames x BT tones (BT = 128 or 64, the tone-tile width chosen by
// the plan's autotuner), K-blocks of 64 complex taps (one plane per TMA
// stage: A hi, lo 128x64 and B hi, lo BTx64, B lo right after B hi).  Per 16
// taps two MMAs: A hi times [B hi | B lo] as one N = 2 BT product (the hi.hi
// and hi.lo terms side by side in TMEM), then A lo times B hi (N = BT) added
// onto the hi.hi half.  The three products of an accumulation chunk run one
// after the other, each into a 2 BT-column TMEM slot taken in rotation (two
// slots for BT = 128, four for 64), so the epilogue drains a slot while the
// MMAs fill the next.  Sixteen epilogue warps (four per TMEM lane quadrant,
// BT/4 tones each) drain a slot by adding its two halves, then add 2 P1 to
// both sums, P2 to the imaginary and -P3 to the real sum.
//
// Fused pre-split (FUSED): instead of TMA loads of the six pre-split source
// planes (written to HBM by presplit3_kernel, 12 bytes per sample), two
// producer warps read the int16 stream view [carry | buffer] and write each
// stage's A hi/lo tiles themselves, in the 128-byte swizzled layout the TMA
// would produce, with the same FP32 -> FP16 hi/lo rounding as the pre-split
// kernel (bit-identical planes, so bit-identical results); only the B tiles
// arrive by TMA.  A launch choice the autotuner times.
//
// The kernel is persistent over a list of plans: one launch runs the tiles
// of every demodulation stream of a batched step (or of one push), each CTA
// striding over the global tile index; a tile's plan is found from the
// plans' first-tile offsets.  Each output element is accumulated in the same
// order whatever the tile width or the plans sharing the launch.
constexpr int G3_BK = 64;                                  // complex taps per K-block
constexpr uint32_t G3_A_BYTES = BM * G3_BK * 2;
constexpr uint32_t G3_A_HALF = G3_A_BYTES / 2;              // 64 rows: one CTA's share in the pair form
constexpr int G3_SLOTS_MAX = 4;
constexpr int G3_EPI_WARPS = 16;          // 4 lane quadrants x 4 tone groups
constexpr int G3_THREADS = (G3_EPI_WARPS + 2) * 32;
constexpr int G3_FUSED_PRODUCERS = 2;                       // producer warps of the fused form
constexpr int G3_THREADS_FUSED = (G3_EPI_WARPS + G3_FUSED_PRODUCERS + 1) * 32;
template <int BT> struct G3Cfg {
    static constexpr uint32_t B_BYTES = BT * G3_BK * 2;
    static constexpr uint32_t STAGE_BYTES = 2 * G3_A_BYTES + 2 * B_BYTES;
    static constexpr int STAGES = BT == 128 ? 3 : 4;
    static constexpr size_t SMEM = 1024 + STAGES * STAGE_BYTES + 256;
    // a slot holds one product's accumulator as two BT-column halves:
    // [0, BT) collects hi.hi + lo.hi, [BT, 2 BT) hi.lo (see the MMA issuer)
    static constexpr int SLOTS = BT == 128 ? 2 : 4;
    static constexpr uint32_t SLOT_COLS = 2 * BT;
    static constexpr uint32_t TMEM_COLS = SLOTS * SLOT_COLS;   // 512
    static constexpr int TPG = BT / 4;                     // tones per epilogue warp
};

struct G3Plan {
    CUtensorMap a[6];   // (x sum/2, xr, xi) x (hi, lo): [rows][D] fp16, Toeplitz view (unused when fused)
    CUtensorMap b[6];   // (cr, ci - cr, cr + ci) x (hi, lo): [ntp][Lpad] fp16, K-major
    GemmArgs g;
    int tile0;          // first global tile of this plan
    // fused form: the int16 stream view v[s] = s < cl ? carry[s] : buf[s - cl]
    // for s < lv (0 beyond); vec: the buffer part may be read 16 bytes at a time
    const uint32_t* carry;
    const uint32_t* buf;
    int64_t cl, lv;
    int vec;
};
constexpr int kG3MaxPlans = 16;
struct G3Batch {
    int n_plans, total_tiles;
    G3Plan p[kG3MaxPlans];
};
static_assert(sizeof(G3Batch) <= 32000, "kernel parameter space");
static_assert(sizeof(G3Plan) <= kDemodJobBytes, "job storage");

__device__ __forceinline__ int g3_plan_of(const G3Batch& bt, int tile) {
    int pi = 0;
    while (pi + 1 < bt.n_plans && tile >= bt.p[pi + 1].tile0) ++pi;
    return pi;
}

// Tile (frame tile mt, tone tile nt) of work item `tile` of a plan.  In the
// pair form a work item is a frame tile and a pair of tone tiles 2j, 2j + 1,
// the CTA of cluster rank r taking tone tile 2j + r (past the plan's last
// tone tile when its count is odd: the taps there are read as zeros and
// no output is stored).
template <bool PAIR>
__device__ __forceinline__ void g3_coords(const GemmArgs& g, int tile, int rank, int& mt, int& nt) {
    if (PAIR) {
        tile_coords_of(g.raster, g.n_mt, (g.n_nt + 1) >> 1, tile, mt, nt);
        nt = 2 * nt + rank;
    } else {
        tile_coords(g, tile, mt, nt);
    }
}

__global__ void build_taps3_kernel(const double* __restrict__ h, const uint64_t* __restrict__ words,
                                   int n_tones, int ntp, int L, int Lpad, double scale,
                                   __half* __restrict__ planes) {
    const int64_t total = static_cast<int64_t>(ntp) * Lpad;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int t = static_cast<int>(idx / Lpad);
        const int n = static_cast<int>(idx - static_cast<int64_t>(t) * Lpad);
        double cr = 0.0, ci = 0.0;
        if (t < n_tones && n < L) {
            const uint64_t ph = words[t] * static_cast<uint64_t>(n);
            const double xs = static_cast<double>(static_cast<int64_t>(ph)) * 0x1p-63;
            double sn, cs;
            sincospi(xs, &sn, &cs);
            const double a = h[n] * scale;
            cr = a * cs;
            ci = -a * sn;
        }
        const double v[3] = {cr, ci - cr, cr + ci};
#pragma unroll
        for (int q = 0; q < 3; ++q) split_store(planes + (2 * q) * total, planes + (2 * q + 1) * total, idx, v[q]);
    }
}

// Sample s of [carry | buffer] -> the six planes ((xr+xi)/2, xr, xi) x (hi, lo).
__global__ void presplit3_kernel(const uint32_t* __restrict__ carry, int64_t cl, const uint32_t* __restrict__ buf,
                                 int64_t lv, int64_t total, __half* __restrict__ planes) {
    for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < total;
         s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint32_t w = 0;
        if (s < lv) w = s < cl ? carry[s] : buf[s - cl];
        const float2 f = iq_to_f2(w);
        const float v[3] = {0.5f * (f.x + f.y), f.x, f.y};      // exact in FP32
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const __half hv = __float2half_rn(v[q]);
            planes[(2 * q) * total + s] = hv;
            planes[(2 * q + 1) * total + s] = __float2half_rn(v[q] - __half2float(hv));
        }
    }
}

// One row (frame m) of a stage's A hi/lo tiles in the fused form: view
// samples s0 .. s0+63 -> plane q ((xr+xi)/2, xr or xi) -> FP16 hi/lo, eight
// samples (one 16-byte chunk) at a time, chunk c of row i stored at
// i*128 + ((c ^ (i & 7)) << 4) (the 128-byte swizzle).
__device__ __forceinline__ void g3_fill_row(const G3Plan& P, int q, int64_t s0, unsigned char* ahi,
                                            unsigned char* alo, int i) {
    const bool in_buf = P.vec && s0 >= P.cl && s0 + G3_BK <= P.lv;
    const uint32_t* bp = P.buf + (s0 - P.cl);
#pragma unroll 2
    for (int c = 0; c < G3_BK / 8; ++c) {
        uint32_t w[8];
        if (in_buf) {
            const uint4 u0 = __ldg(reinterpret_cast<const uint4*>(bp + c * 8));
            const uint4 u1 = __ldg(reinterpret_cast<const uint4*>(bp + c * 8 + 4));
            w[0] = u0.x; w[1] = u0.y; w[2] = u0.z; w[3] = u0.w;
            w[4] = u1.x; w[5] = u1.y; w[6] = u1.z; w[7] = u1.w;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t sv = s0 + c * 8 + e;
                w[e] = sv < P.lv ? (sv < P.cl ? __ldg(P.carry + sv) : __ldg(P.buf + (sv - P.cl))) : 0u;
            }
        }
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const float2 f0 = iq_to_f2(w[e]), f1 = iq_to_f2(w[e + 1]);
            const float v0 = q == 0 ? 0.5f * (f0.x + f0.y) : (q == 1 ? f0.x : f0.y);   // exact in FP32
            const float v1 = q == 0 ? 0.5f * (f1.x + f1.y) : (q == 1 ? f1.x : f1.y);
            const __half h0 = __float2half_rn(v0), h1 = __float2half_rn(v1);
            const __half l0 = __float2half_rn(v0 - __half2float(h0));
            const __half l1 = __float2half_rn(v1 - __half2float(h1));
            hi[e / 2] = static_cast<uint32_t>(__half_as_ushort(h0)) | (static_cast<uint32_t>(__half_as_ushort(h1)) << 16);
            lo[e / 2] = static_cast<uint32_t>(__half_as_ushort(l0)) | (static_cast<uint32_t>(__half_as_ushort(l1)) << 16);
        }
        const uint32_t off = static_cast<uint32_t>(i) * 128u + (static_cast<uint32_t>(c ^ (i & 7)) << 4);
        *reinterpret_cast<uint4*>(ahi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(alo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// PAIR: launched in clusters of two CTAs that take the two tone tiles of a
// work item; they need the same A tiles, so each CTA loads 64 rows of every
// A tile and multicasts them into both CTAs' stage buffers.  A stage of a
// CTA is then refilled only when both CTAs' MMAs have consumed it (its empty
// barrier takes one commit from each), and the two CTAs meet at cluster
// barriers after initialising their mbarriers and before leaving.
template <int BT, bool FUSED, bool PAIR>
__global__ void __launch_bounds__(FUSED ? G3_THREADS_FUSED : G3_THREADS, 1)
demod3m_gemm_kernel(const __grid_constant__ G3Batch bt) {
    static_assert(!(FUSED && PAIR), "the pair form loads its A tiles by TMA");
    using Cfg = G3Cfg<BT>;
    constexpr int STAGES = Cfg::STAGES;
    constexpr uint32_t STAGE_BYTES = Cfg::STAGE_BYTES, B_BYTES = Cfg::B_BYTES;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* sfull = empty + STAGES;
    uint64_t* sempty = sfull + G3_SLOTS_MAX;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(sempty + G3_SLOTS_MAX);
    constexpr int SLOTS = Cfg::SLOTS;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    int* const status0 = bt.p[0].g.status;
    constexpr int PROD_WARP = G3_EPI_WARPS;                                  // first producer warp
    constexpr int MMA_WARP = G3_EPI_WARPS + (FUSED ? G3_FUSED_PRODUCERS : 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rank = PAIR ? static_cast<int>(cluster_ctarank()) : 0;
    const int cta0 = PAIR ? static_cast<int>(blockIdx.x >> 1) : static_cast<int>(blockIdx.x);
    const int ncta = PAIR ? static_cast<int>(gridDim.x >> 1) : static_cast<int>(gridDim.x);
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], FUSED ? G3_FUSED_PRODUCERS * 32 : 1);
            mbar_init(&empty[s], PAIR ? 2 : 1);
        }
        for (int b = 0; b < SLOTS; ++b) {
            mbar_init(&sfull[b], 1);
            mbar_init(&sempty[b], G3_EPI_WARPS * 32);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == MMA_WARP) {
        umma::alloc(tmem_holder, Cfg::TMEM_COLS);
        umma::relinquish();
    }
    if (warp == PROD_WARP && lane < bt.n_plans) {
        for (int i = 0; i < 6; ++i) {
            if (!FUSED) tma_prefetch_desc(&bt.p[lane].a[i]);
            tma_prefetch_desc(&bt.p[lane].b[i]);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (PAIR) cluster_sync();          // both CTAs' barriers exist before any multicast
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    const int n_tiles = bt.total_tiles;
    constexpr uint32_t IDESC = umma::idesc_f16_f32(BM, BT);
    constexpr uint32_t IDESC_W = umma::idesc_f16_f32(BM, 2 * BT);

    if (FUSED && warp >= PROD_WARP && warp < MMA_WARP) {
        // ------------------------------------------------ fused producers
        const int pt = threadIdx.x - PROD_WARP * 32;                         // 0 .. 63
        uint32_t it = 0;
        bool stop = false;
        for (int tile = cta0; tile < n_tiles && !stop; tile += ncta) {
            const int pi = g3_plan_of(bt, tile);
            const G3Plan& P = bt.p[pi];
            int tm, tn;
            g3_coords<PAIR>(P.g, tile - P.tile0, rank, tm, tn);
            const int m0 = tm * BM, n0 = tn * BT;
            const int64_t D = P.g.two_d;
            for (int kb0 = 0; kb0 < P.g.KB && !stop; kb0 += P.g.kchunk) {
                const int kb1 = min(kb0 + P.g.kchunk, P.g.KB);
                for (int q = 0; q < 3 && !stop; ++q) {
                    for (int kb = kb0; kb < kb1; ++kb, ++it) {
                        const int s = it % STAGES;
                        const uint32_t ph = (it / STAGES) & 1;
                        if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1, status0)) {
                            *abort_flag = 1;
                            stop = true;
                            break;
                        }
                        unsigned char* st = smem + s * STAGE_BYTES;
                        const int kt = kb * G3_BK;
                        if (pt == 0) {
                            mbar_expect_tx(&full[s], 2 * B_BYTES);
                            tma_load_2d(st + 2 * G3_A_BYTES, &P.b[2 * q], kt, n0, &full[s]);
                            tma_load_2d(st + 2 * G3_A_BYTES + B_BYTES, &P.b[2 * q + 1], kt, n0, &full[s]);
                        }
#pragma unroll 1
                        for (int i = pt; i < BM; i += G3_FUSED_PRODUCERS * 32)
                            g3_fill_row(P, q, (static_cast<int64_t>(m0) + i) * D + kt, st, st + G3_A_BYTES, i);
                        fence_proxy_async_smem();                 // the MMAs read the tiles through the async proxy
                        mbar_arrive(&full[s]);
                    }
                }
            }
        }
        // the B copies still in flight complete before the CTA exits
        if (pt == 0) {
            for (uint32_t k = 0; k < static_cast<uint32_t>(STAGES) && it > 0; ++k) {
                const uint32_t j = it - 1 - k;
                if (static_cast<int32_t>(j) < 0) break;
                mbar_wait(&full[j % STAGES], (j / STAGES) & 1, status0);
            }
        }
    } else if (!FUSED && warp == PROD_WARP) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            bool stop = false;
            for (int tile = cta0; tile < n_tiles && !stop; tile += ncta) {
                const int pi = g3_plan_of(bt, tile);
                const G3Plan& P = bt.p[pi];
                int tm, tn;
                g3_coords<PAIR>(P.g, tile - P.tile0, rank, tm, tn);
                const int m0 = tm * BM, n0 = tn * BT;
                for (int kb0 = 0; kb0 < P.g.KB && !stop; kb0 += P.g.kchunk) {
                    const int kb1 = min(kb0 + P.g.kchunk, P.g.KB);
                    for (int q = 0; q < 3 && !stop; ++q) {
                        for (int kb = kb0; kb < kb1; ++kb, ++it) {
                            const int s = it % STAGES;
                            const uint32_t ph = (it / STAGES) & 1;
                            if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1, status0)) {
                                *abort_flag = 1;
                                stop = true;
                                break;
                            }
                            unsigned char* st = smem + s * STAGE_BYTES;
                            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                            const int kt = kb * G3_BK;
                            const int c0 = kt % P.g.two_d, c1 = m0 + kt / P.g.two_d;
                            if (PAIR) {
                                // rows 64 r .. 64 r + 63 of both A planes, into both CTAs (64-row boxes)
                                const uint32_t ho = static_cast<uint32_t>(rank) * G3_A_HALF;
                                const int r1 = c1 + rank * (BM / 2);
                                tma_load_2d_mc(st + ho, &P.a[2 * q], c0, r1, &full[s], 0x3);
                                tma_load_2d_mc(st + G3_A_BYTES + ho, &P.a[2 * q + 1], c0, r1, &full[s], 0x3);
                            } else {
                                tma_load_2d(st, &P.a[2 * q], c0, c1, &full[s]);
                                tma_load_2d(st + G3_A_BYTES, &P.a[2 * q + 1], c0, c1, &full[s]);
                            }
                            tma_load_2d(st + 2 * G3_A_BYTES, &P.b[2 * q], kt, n0, &full[s]);
                            tma_load_2d(st + 2 * G3_A_BYTES + B_BYTES, &P.b[2 * q + 1], kt, n0, &full[s]);
                        }
                    }
                }
            }
            // wait for the copies still in flight before leaving
            for (uint32_t k = 0; k < static_cast<uint32_t>(STAGES) && it > 0; ++k) {
                const uint32_t j = it - 1 - k;
                if (static_cast<int32_t>(j) < 0) break;
                mbar_wait(&full[j % STAGES], (j / STAGES) & 1, status0);
            }
            // pair form: and for both CTAs' last commits to this CTA's empty
            // barriers, so that nothing arrives here after the CTA has left
            for (uint32_t k = 0; PAIR && k < static_cast<uint32_t>(STAGES) && it > 0; ++k) {
                const uint32_t j = it - 1 - k;
                if (static_cast<int32_t>(j) < 0) break;
                mbar_wait(&empty[j % STAGES], (j / STAGES) & 1, status0);
            }
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t it = 0, phase = 0;
            bool stop = false;
            for (int tile = cta0; tile < n_tiles && !stop; tile += ncta) {
                const GemmArgs& g = bt.p[g3_plan_of(bt, tile)].g;
                for (int kb0 = 0; kb0 < g.KB && !stop; kb0 += g.kchunk) {
                    const int kb1 = min(kb0 + g.kchunk, g.KB);
                    for (int q = 0; q < 3 && !stop; ++q, ++phase) {
                        const uint32_t slot = phase % SLOTS, use = phase / SLOTS;
                        if (*abort_flag || !mbar_wait(&sempty[slot], (use & 1) ^ 1, status0)) {
                            *abort_flag = 1;
                            stop = true;
                            break;
                        }
                        umma::fence_after_sync();
                        const uint32_t d_tmem = tmem + slot * Cfg::SLOT_COLS;
                        for (int kb = kb0; kb < kb1; ++kb, ++it) {
                            const int s = it % STAGES;
                            const uint32_t ph = (it / STAGES) & 1;
                            if (!mbar_wait(&full[s], ph, status0)) {
                                *abort_flag = 1;
                                stop = true;
                                break;
                            }
                            umma::fence_after_sync();
                            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                            const uint32_t ah = sa, al = sa + G3_A_BYTES;
                            const uint32_t bh = sa + 2 * G3_A_BYTES, bl = bh + B_BYTES;
#pragma unroll
                            for (int k = 0; k < G3_BK / 16; ++k) {
                                const uint32_t off = k * 32;
                                const uint32_t acc = (kb > kb0 || k > 0) ? 1u : 0u;
                                // hi.hi | hi.lo over 2 BT columns (B lo follows B hi), then lo.hi
                                umma::mma_f16(d_tmem, umma::desc_k_sw128(ah + off), umma::desc_k_sw128(bh + off), IDESC_W, acc);
                                umma::mma_f16(d_tmem, umma::desc_k_sw128(al + off), umma::desc_k_sw128(bh + off), IDESC, 1u);
                            }
                            if (PAIR)
                                umma::commit_mc(&empty[s], 0x3);      // frees the stage in both CTAs
                            else
                                umma::commit(&empty[s]);
                        }
                        umma::commit(&sfull[slot]);
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp < G3_EPI_WARPS) {
        // ------------------------------------------------ epilogue (16 warps)
        constexpr int TPG = Cfg::TPG;
        const int qd = warp & 3, grp = warp >> 2;          // lane quadrant, tone group
        const int row = qd * 32 + lane;
        uint32_t phase = 0;
        bool ok = true;
        for (int tile = cta0; tile < n_tiles && ok; tile += ncta) {
            const G3Plan& P = bt.p[g3_plan_of(bt, tile)];
            const GemmArgs& g = P.g;
            int mt, tn;
            g3_coords<PAIR>(g, tile - P.tile0, rank, mt, tn);
            const int m0 = mt * BM, n0 = tn * BT;
            float re[TPG], im[TPG];
#pragma unroll
            for (int i = 0; i < TPG; ++i) re[i] = im[i] = 0.f;
            for (int kb0 = 0; kb0 < g.KB && ok; kb0 += g.kchunk) {
                for (int q = 0; q < 3; ++q, ++phase) {
                    const uint32_t slot = phase % SLOTS, use = phase / SLOTS;
                    if (*abort_flag || !mbar_wait(&sfull[slot], use & 1, status0)) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    umma::fence_after_sync();
                    const uint32_t ta = tmem + (static_cast<uint32_t>(qd * 32) << 16) + slot * Cfg::SLOT_COLS + grp * TPG;
                    // the product = (hi.hi + lo.hi) + hi.lo, 16 tones at a time
#pragma unroll
                    for (int h = 0; h < TPG; h += 16) {
                        uint32_t r0[16], r1[16];
                        umma::ld_32x32b_x16(ta + h, r0);
                        umma::ld_32x32b_x16(ta + BT + h, r1);
                        umma::wait_ld_regs(r0);
                        umma::wait_ld_regs(r1);
                        float pv[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) pv[i] = __uint_as_float(r0[i]) + __uint_as_float(r1[i]);
                        if (q == 0) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const float v = 2.f * pv[i];
                                re[h + i] += v;
                                im[h + i] += v;
                            }
                        } else if (q == 1) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) im[h + i] += pv[i];
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i) re[h + i] -= pv[i];
                        }
                    }
                    umma::fence_before_sync();
                    mbar_arrive(&sempty[slot]);
                }
            }
            if (!ok) break;
            const int64_t k = static_cast<int64_t>(m0) + row;
            if (k < g.F) {
                const int tb = n0 + grp * TPG;
                const int64_t K = g.F0 + k;
                const int64_t arow = K / BM - g.F0 / BM;
                const int si = static_cast<int>(K % BM);
#pragma unroll
                for (int tl = 0; tl < TPG; ++tl) {
                    const int t = tb + tl;
                    if (t < g.n_tones) {
                        const float2 an = __ldg(g.anchors + arow * g.ntp + t);
                        const float2 sp = __ldg(g.steps + static_cast<int64_t>(t) * BM + si);
                        const float2 rot = cmul(an, sp);
                        const float2 acc = make_float2(re[tl] * g.inv_scale, im[tl] * g.inv_scale);
                        g.out[static_cast<int64_t>(t) * g.ld + g.fo + k] = cmul(acc, rot);
                    }
                }
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (PAIR) cluster_sync();          // neither CTA leaves while the other may still signal it
    if (warp == MMA_WARP) {
        umma::fence_after_sync();
        umma::dealloc(tmem, Cfg::TMEM_COLS);
    }
}

// ------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tmap_encode_tiled_fn());
}

// 2-D fp16 tensor [rows][cols] (cols contiguous), box [box_rows][64], 128B swizzle.
bool make_map(CUtensorMap* m, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(BK), box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

unsigned grid_for(int64_t work, int n_sms) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, int64_t(n_sms) * 16)));
}

}  // namespace

int demod_anchor_rows(int64_t F0, int64_t F) {
    return static_cast<int>((F0 + F - 1) / BM - F0 / BM + 1);
}

size_t demod_xs_rows(int64_t F, int Lpad, int D) {
    // frame F-1 reads rows F-1 .. F-1 + (Lpad-1)/D
    return static_cast<size_t>(F + (Lpad - 1) / D);
}

size_t demod3_xs_rows(int64_t F, int Lpad, int D) { return static_cast<size_t>(F + (Lpad - 1) / D); }

cudaError_t demod_build_taps(const double* d_h, const uint64_t* d_words, int n_tones, int ntp, int L,
                             int Lpad, int e, void* b_hi, void* b_lo, cudaStream_t st) {
    const int64_t total = static_cast<int64_t>(ntp) * Lpad;
    build_taps_kernel<<<grid_for(total, 152), 256, 0, st>>>(d_h, d_words, n_tones, ntp, L, Lpad,
                                                             std::ldexp(1.0, e), static_cast<__half*>(b_hi),
                                                             static_cast<__half*>(b_lo));
    return cudaGetLastError();
}

cudaError_t demod_launch(const DemodLaunch& L, cudaStream_t st) {
    if (L.F <= 0) return cudaSuccess;
    if (L.D % 32 != 0 || L.Lpad % 32 != 0) return cudaErrorInvalidValue;
    const int64_t rows = static_cast<int64_t>(demod_xs_rows(L.F, L.Lpad, L.D));
    if (rows > L.xs_rows) return cudaErrorInvalidValue;
    const int n_mt = static_cast<int>((L.F + BM - 1) / BM);
    const int n_nt = (2 * L.ntp) / BN;
    const int n_anch = demod_anchor_rows(L.F0, L.F);
    float2* anchors = static_cast<float2*>(L.rot);
    float2* steps = anchors + static_cast<int64_t>(n_anch) * L.ntp;
    // rotation tables
    const int64_t nrot = static_cast<int64_t>(n_anch) * L.ntp + static_cast<int64_t>(L.ntp) * BM;
    rot_kernel<<<grid_for(nrot, L.n_sms), 256, 0, st>>>(L.words, L.n_tones, L.ntp, L.F0 / BM, L.L, L.D,
                                                         n_anch, anchors, steps);
    // pre-split of the Toeplitz source rows
    const int64_t total = rows * L.D;
    presplit_kernel<<<grid_for(total, L.n_sms), 256, 0, st>>>(
        reinterpret_cast<const uint32_t*>(L.carry), L.cl, reinterpret_cast<const uint32_t*>(L.buf),
        L.cl + L.n, total, static_cast<__half2*>(L.xs_hi), static_cast<__half2*>(L.xs_lo));
    // tensor maps
    CUtensorMap mAh, mAl, mBh, mBl;
    const uint64_t two_d = static_cast<uint64_t>(2) * L.D;
    if (!make_map(&mAh, L.xs_hi, two_d, rows, BM) || !make_map(&mAl, L.xs_lo, two_d, rows, BM) ||
        !make_map(&mBh, L.b_hi, static_cast<uint64_t>(2) * L.Lpad, static_cast<uint64_t>(2) * L.ntp, BN) ||
        !make_map(&mBl, L.b_lo, static_cast<uint64_t>(2) * L.Lpad, static_cast<uint64_t>(2) * L.ntp, BN))
        return cudaErrorInvalidValue;
    GemmArgs g{};
    g.raster = L.raster_group;
    g.F = L.F;
    g.F0 = L.F0;
    g.n_tones = L.n_tones;
    g.ntp = L.ntp;
    g.KB = 2 * L.Lpad / BK;
    g.kchunk = L.kchunk > 0 ? L.kchunk : 2;
    g.two_d = static_cast<int>(two_d);
    g.n_mt = n_mt;
    g.n_nt = n_nt;
    g.anchors = anchors;
    g.steps = steps;
    g.inv_scale = static_cast<float>(L.inv_scale);
    g.out = static_cast<float2*>(L.tones);
    g.ld = L.tones_ld;
    g.fo = L.frame_offset;
    g.status = L.status;
    cudaError_t e = cudaFuncSetAttribute(demod_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(GEMM_SMEM));
    if (e != cudaSuccess) return e;
    const int tiles = n_mt * n_nt;
    const int grid = std::min(tiles, L.n_sms);
    demod_gemm_kernel<<<grid, GEMM_THREADS, GEMM_SMEM, st>>>(mAh, mAl, mBh, mBl, g);
    return cudaGetLastError();
}

cudaError_t demod3_build_taps(const double* d_h, const uint64_t* d_words, int n_tones, int ntp, int L, int Lpad,
                              int e, void* planes, cudaStream_t st) {
    const int64_t total = static_cast<int64_t>(ntp) * Lpad;
    build_taps3_kernel<<<grid_for(total, 152), 256, 0, st>>>(d_h, d_words, n_tones, ntp, L, Lpad, std::ldexp(1.0, e),
                                                              static_cast<__half*>(planes));
    return cudaGetLastError();
}

cudaError_t demod3_prepare(const DemodLaunch& L, cudaStream_t st, DemodGemmJob* job) {
    job->n_tiles = 0;
    job->bt = L.tone_tile == 64 ? 64 : 128;
    job->fused = L.fused_presplit ? 1 : 0;
    job->pair = (L.pair && !job->fused) ? 1 : 0;
    if (L.F <= 0) return cudaSuccess;
    if (L.D % G3_BK != 0 || L.Lpad % G3_BK != 0 || L.ntp % 128 != 0) return cudaErrorInvalidValue;
    const int64_t rows = static_cast<int64_t>(demod3_xs_rows(L.F, L.Lpad, L.D));
    if (!job->fused && rows > L.xs_rows) return cudaErrorInvalidValue;
    const int bt = job->bt;
    const int n_mt = static_cast<int>((L.F + BM - 1) / BM);
    const int n_nt = (L.n_tones + bt - 1) / bt;       // tiles past the last tone are skipped
    const int n_anch = demod_anchor_rows(L.F0, L.F);
    float2* anchors = static_cast<float2*>(L.rot);
    float2* steps = anchors + static_cast<int64_t>(n_anch) * L.ntp;
    const int64_t nrot = static_cast<int64_t>(n_anch) * L.ntp + static_cast<int64_t>(L.ntp) * BM;
    rot_kernel<<<grid_for(nrot, L.n_sms), 256, 0, st>>>(L.words, L.n_tones, L.ntp, L.F0 / BM, L.L, L.D, n_anch,
                                                         anchors, steps);
    G3Plan* P = reinterpret_cast<G3Plan*>(job->bytes);
    std::memset(P, 0, sizeof(G3Plan));
    const __half* bp = static_cast<const __half*>(L.b_hi);
    const int64_t bplane = static_cast<int64_t>(L.ntp) * L.Lpad;
    const int64_t total = rows * L.D;
    __half* xp = static_cast<__half*>(L.xs_hi);
    if (job->fused) {
        // the GEMM's producers read the stream view themselves
        P->carry = reinterpret_cast<const uint32_t*>(L.carry);
        P->buf = reinterpret_cast<const uint32_t*>(L.buf);
        P->cl = L.cl;
        P->lv = L.cl + L.n;
        P->vec = (reinterpret_cast<uintptr_t>(L.buf) % 16 == 0) && ((L.cl % 4) + 4) % 4 == 0 ? 1 : 0;
    } else {
        presplit3_kernel<<<grid_for(total, L.n_sms), 256, 0, st>>>(
            reinterpret_cast<const uint32_t*>(L.carry), L.cl, reinterpret_cast<const uint32_t*>(L.buf), L.cl + L.n,
            total, xp);
    }
    for (int i = 0; i < 6; ++i) {
        if ((!job->fused && !make_map(&P->a[i], xp + i * total, static_cast<uint64_t>(L.D),
                                      static_cast<uint64_t>(rows), job->pair ? BM / 2 : BM)) ||
            !make_map(&P->b[i], bp + i * bplane, static_cast<uint64_t>(L.Lpad), static_cast<uint64_t>(L.ntp), bt))
            return cudaErrorInvalidValue;
    }
    GemmArgs& g = P->g;
    g.raster = L.raster_group;
    g.F = L.F;
    g.F0 = L.F0;
    g.n_tones = L.n_tones;
    g.ntp = L.ntp;
    g.KB = L.Lpad / G3_BK;
    g.kchunk = L.kchunk > 0 ? L.kchunk : 1;
    g.two_d = L.D;                 // columns of a Toeplitz source row (one plane)
    g.n_mt = n_mt;
    g.n_nt = n_nt;
    g.anchors = anchors;
    g.steps = steps;
    g.inv_scale = static_cast<float>(L.inv_scale);
    g.out = static_cast<float2*>(L.tones);
    g.ld = L.tones_ld;
    g.fo = L.frame_offset;
    g.status = L.status;
    job->n_tiles = n_mt * (job->pair ? (n_nt + 1) / 2 : n_nt);
    return cudaGetLastError();
}

namespace {
template <int BT, bool FUSED, bool PAIR>
cudaError_t g3_run(const G3Batch& b, int n_sms, cudaStream_t st) {
    using Cfg = G3Cfg<BT>;
    auto kern = demod3m_gemm_kernel<BT, FUSED, PAIR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(Cfg::SMEM));
    if (e != cudaSuccess) return e;
    const int threads = FUSED ? G3_THREADS_FUSED : G3_THREADS;
    if (!PAIR) {
        const int grid = std::max(1, std::min(b.total_tiles, n_sms));
        kern<<<grid, threads, Cfg::SMEM, st>>>(b);
        return cudaGetLastError();
    }
    // clusters of two CTAs: as many as can be resident at once (one CTA per SM)
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = Cfg::SMEM;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static int max_clusters[2] = {0, 0};          // per tile width, queried once
    int& mc = max_clusters[BT == 128 ? 0 : 1];
    if (mc <= 0) {
        cfg.gridDim = dim3(static_cast<unsigned>(2 * (n_sms / 2)), 1, 1);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = n_sms / 2;
        }
        mc = n;
    }
    const int clusters = std::max(1, std::min(b.total_tiles, mc));
    cfg.gridDim = dim3(static_cast<unsigned>(2 * clusters), 1, 1);
    e = cudaLaunchKernelEx(&cfg, kern, b);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
}  // namespace

cudaError_t demod3_gemm(const DemodGemmJob* const* jobs, int n, int n_sms, cudaStream_t st) {
    // one persistent launch per group of up to kG3MaxPlans jobs of the same
    // tile width, producer form and cluster form
    for (int variant = 0; variant < 8; ++variant) {
        const int bt = variant & 1 ? 64 : 128;
        const int fused = (variant >> 1) & 1;
        const int pair = variant >> 2;
        if (fused && pair) continue;
        G3Batch b;
        b.n_plans = 0;
        b.total_tiles = 0;
        for (int i = 0; i <= n; ++i) {
            const bool flush = i == n || b.n_plans == kG3MaxPlans;
            if (flush && b.n_plans > 0) {
                cudaError_t e;
                if (pair)
                    e = bt == 128 ? g3_run<128, false, true>(b, n_sms, st) : g3_run<64, false, true>(b, n_sms, st);
                else if (fused)
                    e = bt == 128 ? g3_run<128, true, false>(b, n_sms, st) : g3_run<64, true, false>(b, n_sms, st);
                else
                    e = bt == 128 ? g3_run<128, false, false>(b, n_sms, st) : g3_run<64, false, false>(b, n_sms, st);
                if (e != cudaSuccess) return e;
                b.n_plans = 0;
                b.total_tiles = 0;
            }
            if (i == n) break;
            if (jobs[i]->bt != bt || jobs[i]->fused != fused || jobs[i]->pair != pair || jobs[i]->n_tiles <= 0)
                continue;
            std::memcpy(&b.p[b.n_plans], jobs[i]->bytes, sizeof(G3Plan));
            b.p[b.n_plans].tile0 = b.total_tiles;
            b.total_tiles += jobs[i]->n_tiles;
            ++b.n_plans;
        }
    }
    return cudaSuccess;
}

cudaError_t demod3_launch(const DemodLaunch& L, cudaStream_t st) {
    DemodGemmJob job;
    cudaError_t e = demod3_prepare(L, st, &job);
    if (e != cudaSuccess || job.n_tiles <= 0) return e;
    const DemodGemmJob* jp = &job;
    return demod3_gemm(&jp, 1, L.n_sms, st);
}

}  // namespace rfr

// ====================================================================
// Allocation-free one-shot demodulation (rfr_demod_noalloc).
//
// For callers that must not allocate device memory once they are running:
// a real-time processing thread that cannot afford the device-wide
// synchronisation and allocator locks that cudaMalloc/cudaFree can take, or a
// host application whose device-memory budget is owned by another allocator.
// The working memory of this path -- the modulated taps, the FP16 split of
// the samples, the rotation tables, a zero history block and the status word
// -- lives in one file-scope device array of kNaBytes (about 6.7 MB), which
// every GPU that loads this library holds until the process exits.
// ====================================================================
#include <mutex>

namespace rfr {
namespace {

constexpr int64_t kNaMaxSamples = int64_t(1) << 18;   // samples per call
constexpr int kNaMaxTones = 256;
constexpr int kNaMaxTaps = 1024;

constexpr size_t na_align(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kNaStatus = 0;
constexpr size_t kNaWords = 256;
constexpr size_t kNaTaps = na_align(kNaWords + kNaMaxTones * 8);
constexpr size_t kNaZero = na_align(kNaTaps + kNaMaxTaps * 8);                 // zero history
constexpr size_t kNaBhi = na_align(kNaZero + kNaMaxTaps * 4);
constexpr size_t kNaBBytes = static_cast<size_t>(2) * kNaMaxTones * 2 * kNaMaxTaps * 2;
constexpr size_t kNaBlo = na_align(kNaBhi + kNaBBytes);
constexpr size_t kNaXsBytes = static_cast<size_t>(kNaMaxSamples + kNaMaxTaps) * 4;
constexpr size_t kNaXhi = na_align(kNaBlo + kNaBBytes);
constexpr size_t kNaXlo = na_align(kNaXhi + kNaXsBytes);
constexpr int64_t kNaMaxAnchRows = kNaMaxSamples / 32 / BM + 2;
constexpr size_t kNaRot = na_align(kNaXlo + kNaXsBytes);
constexpr size_t kNaRotBytes = static_cast<size_t>(kNaMaxAnchRows + BM) * kNaMaxTones * 8;
constexpr size_t kNaBytes = na_align(kNaRot + kNaRotBytes);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of g_noalloc_scratch per device, looked up once per device
// (the host-side name of the array is not a device address).
constexpr int kNaMaxDevices = 64;
unsigned char* g_na_ptr[kNaMaxDevices] = {};
std::mutex g_na_mu;

cudaError_t na_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace rfr

extern "C" rfr_status rfr_demod_noalloc(const int16_t* iq, int64_t n_samples, const double* taps,
                                        int32_t L, int32_t D, const uint64_t* words, int32_t n_tones,
                                        void* tones, int64_t tones_ld, void* stream) {
    using namespace rfr;
    if (n_samples < 0 || n_samples > kNaMaxSamples) return RFR_E_INVALID;   // beyond the static scratch
    if (L < 1 || L > kNaMaxTaps || D < 32 || D % 32 != 0 || D > kNaMaxSamples) return RFR_E_INVALID;
    if (n_tones < 1 || n_tones > kNaMaxTones || !taps || !words) return RFR_E_INVALID;
    const int64_t F = n_samples / D;
    if (F > 0 && (!iq || !tones || tones_ld < F)) return RFR_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* base = nullptr;
    if (na_scratch(&base) != cudaSuccess) return RFR_E_CUDA;
    if (F == 0) return RFR_OK;
    // tap scale 2^e with max|h| * 2^e in [2^14, 2^15) (same rule as a plan)
    double hmax = 0.0;
    for (int j = 0; j < L; ++j) hmax = std::max(hmax, std::fabs(taps[j]));
    if (!(hmax > 0.0) || !std::isfinite(hmax)) return RFR_E_INVALID;
    int e2 = 0;
    std::frexp(hmax, &e2);
    const int tap_exp = 15 - e2;
    const int Lpad = (L + 31) / 32 * 32;
    const int ntp = (n_tones + BN / 2 - 1) / (BN / 2) * (BN / 2);
    int* status = reinterpret_cast<int*>(base + kNaStatus);
    uint64_t* d_words = reinterpret_cast<uint64_t*>(base + kNaWords);
    double* d_taps = reinterpret_cast<double*>(base + kNaTaps);
    const uint32_t* zero = reinterpret_cast<const uint32_t*>(base + kNaZero);
    __half* bh = reinterpret_cast<__half*>(base + kNaBhi);
    __half* bl = reinterpret_cast<__half*>(base + kNaBlo);
    __half2* xh = reinterpret_cast<__half2*>(base + kNaXhi);
    __half2* xl = reinterpret_cast<__half2*>(base + kNaXlo);
    float2* anchors = reinterpret_cast<float2*>(base + kNaRot);
    // contents left by the previous call are overwritten or cleared here
    if (cudaMemsetAsync(base, 0, kNaTaps, st) != cudaSuccess ||
        cudaMemsetAsync(base + kNaZero, 0, static_cast<size_t>(kNaMaxTaps) * 4, st) != cudaSuccess ||
        cudaMemcpyAsync(d_words, words, static_cast<size_t>(n_tones) * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_taps, taps, static_cast<size_t>(L) * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return RFR_E_CUDA;
    build_taps_kernel<<<grid_for(static_cast<int64_t>(ntp) * Lpad, 152), 256, 0, st>>>(
        d_taps, d_words, n_tones, ntp, L, Lpad, std::ldexp(1.0, tap_exp), bh, bl);
    const int n_mt = static_cast<int>((F + BM - 1) / BM);
    const int n_anch = demod_anchor_rows(0, F);
    float2* steps = anchors + static_cast<int64_t>(n_anch) * ntp;
    rot_kernel<<<grid_for(static_cast<int64_t>(n_anch + BM) * ntp, 152), 256, 0, st>>>(
        d_words, n_tones, ntp, 0, L, D, n_anch, anchors, steps);
    // zero history: the stream view starts L - D samples before sample 0
    const int64_t cl = static_cast<int64_t>(L) - D;
    const int64_t rows = static_cast<int64_t>(demod_xs_rows(F, Lpad, D));
    presplit_kernel<<<grid_for(rows * D, 152), 256, 0, st>>>(zero, cl, reinterpret_cast<const uint32_t*>(iq),
                                                             cl + n_samples, rows * D, xh, xl);
    CUtensorMap mAh, mAl, mBh, mBl;
    const uint64_t two_d = static_cast<uint64_t>(2) * D;
    if (!make_map(&mAh, xh, two_d, rows, BM) || !make_map(&mAl, xl, two_d, rows, BM) ||
        !make_map(&mBh, bh, static_cast<uint64_t>(2) * Lpad, static_cast<uint64_t>(2) * ntp, BN) ||
        !make_map(&mBl, bl, static_cast<uint64_t>(2) * Lpad, static_cast<uint64_t>(2) * ntp, BN))
        return RFR_E_CUDA;
    GemmArgs g{};
    g.raster = 1;
    g.F = F;
    g.F0 = 0;
    g.n_tones = n_tones;
    g.ntp = ntp;
    g.KB = 2 * Lpad / BK;
    g.kchunk = 2;
    g.two_d = static_cast<int>(two_d);
    g.n_mt = n_mt;
    g.n_nt = (2 * ntp) / BN;
    g.anchors = anchors;
    g.steps = steps;
    g.inv_scale = static_cast<float>(std::ldexp(1.0, -tap_exp));
    g.out = static_cast<float2*>(tones);
    g.ld = tones_ld;
    g.fo = 0;
    g.status = status;
    if (cudaFuncSetAttribute(demod_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(GEMM_SMEM)) != cudaSuccess)
        return RFR_E_CUDA;
    int n_sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
    demod_gemm_kernel<<<std::min(n_mt * g.n_nt, std::max(n_sms, 1)), GEMM_THREADS, GEMM_SMEM, st>>>(mAh, mAl, mBh, mBl, g);
    return cudaGetLastError() == cudaSuccess ? RFR_OK : RFR_E_CUDA;
}

extern "C" rfr_status rfr_demod_noalloc_status(void* stream, int32_t* device_status) {
    using namespace rfr;
    unsigned char* base = nullptr;
    if (na_scratch(&base) != cudaSuccess) return RFR_E_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int v = 0;
    if (cudaMemcpyAsync(&v, base + kNaStatus, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RFR_E_CUDA;
    if (device_status) *device_status = v;
    if (v == DEV_TIMEOUT) return RFR_E_TIMEOUT;
    return v == DEV_OK ? RFR_OK : RFR_E_CUDA;
}
