// rfr_internal.h -- internal structures of the readout library (not part of
// the ABI).  The plan holds the host-built coefficient tables (FP64), their
// device copies, the stream state kept on the device across pushes, and
// cached scratch buffers.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rfr.h"

namespace rfr {

// ------------------------------------------------------------ host tables
// Window and prototype builders (FP64), written from the definitions in
// Sec. III.A/B; see plan_host.cpp.
int build_window(int kind, double beta, int64_t m, double* w);
int build_lowpass(int kind, double beta, double fc, int64_t m, double* h);
uint64_t freq_to_word(double f, double fs);
int32_t word_to_bin(uint64_t word, int32_t n);

// --------------------------------------------------------------- PFB
struct PfbLaunch {
    const int16_t* carry;
    int64_t cl;
    const int16_t* buf;
    int64_t n;
    int64_t F;
    int log2n;
    int taps_kernel;
    const float* h;
    const void* tw;
    int tw_count;
    const int32_t* bins;
    int n_tones;
    void* full;
    int64_t full_ld;
    void* tones;
    int64_t tones_ld;
    int64_t frame_offset;
    int* status;
    int n_sms;
    int max_smem;
    int lookahead;      // ring super-blocks fetched ahead (0 = as many as fit, <= 3)
    int variant;        // 0 = best available, 1 = shared-memory int16 ring only,
                        // 2 = no symmetric-tap TMEM kernel
    int sym_taps;       // kernel taps exactly symmetric (h[j] == h[T*N - 1 - j])
    int tone_cs;        // tone columns of consecutive frames this far apart (0/1: adjacent)
    int rot;            // bin c multiplied by (-i)^((c * rot) mod 4) (phase passes)
    int hop;            // samples between frames (N: critically sampled)
    int64_t a0;         // absolute sample index of the virtual stream's first sample
    int cluster;        // N = 8192, 16384 (T <= 8): the cluster kernel instead of the direct one
    const void* tw_cl;  // its twiddles: the 4096-point FFT's, then W_N^(k2 p1)
    int tw_cl_count;    // entries of the 4096-point FFT part
    void* pre;          // FIR pre-sum rows [pre_cap][N] (float2) of pfb_pre_rows plans, or null
    int64_t pre_cap;
};
bool pfb_uses_ring(int log2n, int taps);
// cuTensorMapEncodeTiled (PFN_cuTensorMapEncodeTiled_v12000) or nullptr
void* tmap_encode_tiled_fn();

// PFB for any N = 2^a 3^b 5^c 7^d <= 2^24 (pfb_general.cu): mixed-radix
// in-CTA FFT, one pass for N <= 16384, the four-step split N = N1*N2 above.
constexpr int kGenMaxStages = 24;
struct GenFft {                 // one mixed-radix transform length
    int n = 0;
    int nst = 0;                // stages
    int radix[kGenMaxStages];
    int ns[kGenMaxStages];      // span: product of the earlier radices
    uint32_t ns_magic[kGenMaxStages];   // ceil(2^32 / ns)
    int tw_off[kGenMaxStages];  // offset of the stage's twiddles in the table
};
struct GenPlan {
    int N = 0, N1 = 1, N2 = 0;  // N1 == 1: single pass
    int gla = 0, glb = 0;       // log2 of the transforms per CTA in pass A / B
    int gls = 0;                // one pass: log2 of the frames per CTA iteration
    int threads = 256;          // CTA shape: 256 threads x 4096 points or 512 x 8192
    GenFft fa{}, fb{};          // lengths N1 (pass A) and N2 (pass B / single pass)
    float2* d_tw = nullptr;     // stage twiddles of fa and fb (absolute tw_off)
    float2* d_tw3 = nullptr;    // [3][256]: W_N^i, W_N^(256 i), W_N^(65536 i)
    float2* d_z = nullptr;      // between-pass buffer, z_frames x N
    int64_t z_frames = 0;
    int64_t z_cap_frames = 0;   // the most frames Z grows to
    // pass B's tone lists: the tones of pass-B group i (bins with c1 in
    // [i*GB, (i+1)*GB)) are d_gtone[d_goff[i] .. d_goff[i+1]), each {tone,
    // its index (c2 << glb) + c1 - i*GB in the group's spectrum}
    int2* d_gtone = nullptr;
    int* d_goff = nullptr;
    // vtma: the FIR runs as its own kernel into V (z_frames x N, natural
    // order) and pass A fetches its points by 2-D TMA boxes of V (N2 even,
    // boxes fit the CTA's second buffer); else pass A computes the FIR
    int vtma = 0, vbox_rows = 0, vboxes = 0, vsstride = 0;
    float2* d_v = nullptr;
};
bool gen_supported(int64_t n);
cudaError_t gen_plan_init(GenPlan* g, int N, int64_t z_budget_bytes);
// Grow Z to min(frames, z_cap_frames) (allocates and synchronises the device;
// never during stream capture).
cudaError_t gen_plan_reserve(GenPlan* g, int64_t frames);
// The tone lists of pass B from the tones' bins (two-pass plans; no-op otherwise).
cudaError_t gen_plan_set_tones(GenPlan* g, const int32_t* bins, int n_tones);
void gen_plan_free(GenPlan* g);
int pfb_kernel_taps(int log2n, int taps);
// CTAs per cluster of the cluster PFB kernel (N = 8192, 16384 with T <= 8), else 0.
int pfb_cluster_size(int log2n, int taps);
// N = 4096 with 16 kernel taps: a first-half FIR pass, then the TMEM kernel
// seeded with it (aligned view, PfbLaunch::pre for the frames).
bool pfb_split16(int log2n, int taps);
// PFB plans whose pushes take FIR pre-sum rows (PfbLaunch::pre): the 16-tap
// N = 4096 form and the direct kernel's shapes (N = 8192, 16384; T > 8).
bool pfb_pre_rows(int log2n, int taps);
cudaError_t pfb_launch(const PfbLaunch& L, cudaStream_t st);
cudaError_t gen_pfb_launch(const PfbLaunch& L, const GenPlan& g, cudaStream_t st);

// ------------------------------------------------------------- demod
// Split-FP16 tensor-core demodulation; see demod_*.cu.
constexpr int kDemodBM = 128;         // frames per tile
constexpr int kDemodBN = 256;         // real output columns (= 128 tones) per tile
constexpr int kDemodBK = 64;          // halfs of K per k-block (32 complex taps)

struct DemodLaunch {
    const int16_t* carry;
    int64_t cl;
    const int16_t* buf;
    int64_t n;
    int64_t F;
    int64_t a0;                 // absolute sample index of v[0]
    int64_t F0;                 // frames of the stream before this push
    int32_t L, D, Lpad, n_tones, ntp;   // ntp = tones padded to kDemodBN/2
    const uint64_t* words;      // device [n_tones]
    const void* b_hi;           // device fp16 [2*ntp][2*Lpad]
    const void* b_lo;
    double inv_scale;           // 2^-e
    void* xs_hi;                // scratch fp16 [rows][2*D]
    void* xs_lo;
    int64_t xs_rows;
    void* rot;                  // scratch float2 rotation anchors
    void* tones;
    int64_t tones_ld;
    int64_t frame_offset;
    int* status;
    int n_sms;
    int kchunk;                 // k-blocks per TMEM accumulation chunk
    int raster_group;           // tile order: groups of this many 128-frame tiles sweep all tones
    int tone_tile;              // three-product GEMM: tones per tile, 128 or 64 (0 = 128)
    int fused_presplit;         // three-product GEMM: producers convert the int16 stream themselves
    int pair;                   // three-product GEMM: clusters of two CTAs sharing A tiles by multicast
};
// The three-product GEMM of one push, described for a persistent launch that
// may cover several plans (opaque record of demod.cu).
constexpr int kDemodJobBytes = 2048;
struct DemodGemmJob {
    alignas(128) unsigned char bytes[kDemodJobBytes];
    int bt = 128;               // tone-tile width
    int fused = 0;              // pre-split fused into the GEMM's producers
    int pair = 0;               // two-CTA clusters (n_tiles then counts tone-tile pairs)
    int n_tiles = 0;            // 0: nothing to launch
};
cudaError_t demod_build_taps(const double* d_h, const uint64_t* d_words, int n_tones, int ntp,
                             int L, int Lpad, int e, void* b_hi, void* b_lo, cudaStream_t st);
cudaError_t demod_launch(const DemodLaunch& L, cudaStream_t st);
size_t demod_xs_rows(int64_t F, int Lpad, int D);
// Gauss three-product form: B planes (cr, ci - cr, cr + ci) x (hi, lo), each
// [ntp][Lpad] fp16 (ntp a multiple of 128, Lpad of 64); the launch takes them
// in b_hi, and the six [rows][D] source planes in xs_hi (D % 64 == 0).
cudaError_t demod3_build_taps(const double* d_h, const uint64_t* d_words, int n_tones, int ntp, int L, int Lpad,
                              int e, void* planes, cudaStream_t st);
cudaError_t demod3_launch(const DemodLaunch& L, cudaStream_t st);
// the per-push kernels before the GEMM (rotation tables, pre-split), and the
// GEMM's description in *job
cudaError_t demod3_prepare(const DemodLaunch& L, cudaStream_t st, DemodGemmJob* job);
// persistent GEMM launch(es) over the jobs' tiles (one per tone-tile width
// and per 16 plans)
cudaError_t demod3_gemm(const DemodGemmJob* const* jobs, int n, int n_sms, cudaStream_t st);
size_t demod3_xs_rows(int64_t F, int Lpad, int D);
int demod_anchor_rows(int64_t F0, int64_t F);

// -------------------------------------------------------------- chirp
struct ChirpLaunch {
    const int16_t* carry;
    int64_t cl;
    const int16_t* buf;
    int64_t F;
    int64_t a0;
    int L, D;
    const float* h32;
    const uint64_t* start_words;
    const uint64_t* rate_words;
    int n_chirps;
    void* tones;
    int64_t tones_ld, frame_offset;
    int n_sms;
};
cudaError_t chirp_synth(uint64_t start_word, uint64_t rate_word, double amp, int64_t m0, int64_t n,
                        void* out, cudaStream_t st);
cudaError_t chirp_demod_launch(const ChirpLaunch& L, cudaStream_t st);

// -------------------------------------------------------------- plain
cudaError_t plain_pfb(const int16_t* iq, int64_t n, int N, int T, const float* h, const int32_t* bins,
                      int n_tones, void* full, int64_t full_ld, void* tones, int64_t tones_ld,
                      void** scratch, size_t* scratch_bytes, void** fft_plan, int64_t* fft_batch,
                      cudaStream_t st);
cudaError_t plain_demod_taps(const float* h32, const uint64_t* words, int n_tones, int L, void* c32,
                             cudaStream_t st);
cudaError_t plain_demod(const int16_t* iq, int64_t n, int L, int D, const void* c32,
                        const uint64_t* words, int n_tones, void* tones, int64_t tones_ld,
                        cudaStream_t st);
cudaError_t plain_demod_cgemm(const int16_t* iq, int64_t n, int L, int D, const void* c32,
                              const uint64_t* words, int n_tones, void* tones, int64_t tones_ld,
                              void** scratch, size_t* scratch_bytes, void** blas, cudaStream_t st);
void plain_release(void* scratch, void* fft_plan, void* blas);

// ------------------------------------------------------------- tuning
// Launch choices that never change results (bit-identical outputs).
struct TuneConfig {
    int pfb_lookahead = 0;      // 0 = as many ring super-blocks as shared memory allows
    int demod_raster = 1;       // 1 = tones fastest across the whole grid
    int demod_bt = 128;         // three-product GEMM: tones per tile (128 or 64)
    int demod_fused = 0;        // three-product GEMM: pre-split fused into its producers (0/1)
    int demod_pair = 0;         // three-product GEMM: two-CTA clusters sharing A tiles (0/1)
    int pfb_cluster = 0;        // PFB N = 8192, 16384 with T <= 8: cluster kernel (1) or direct (0)
    bool tuned = false;
};

// ------------------------------------------------------------- state
cudaError_t carry_update(const int16_t* old_carry, int64_t cl, const int16_t* buf, int64_t n,
                         int64_t from, int64_t count, int16_t* new_carry, cudaStream_t st);
// out[t * ld + R m + k] = src[(k * n_tones + t) * src_ld + m] for R m + k < F:
// the R phase passes' tone rows interleaved into [tone][frame].
cudaError_t interleave_tones(const void* src, int64_t src_ld, int R, int n_tones, int64_t F, void* out,
                             int64_t ld, cudaStream_t st);

}  // namespace rfr

// The plan.  Mode-specific members are unused in the other mode.
struct rfr_plan {
    int mode = 0;
    int32_t N = 0, T = 0, Tk = 0, log2n = 0;   // PFB (Tk: kernel taps, zero-padded)
    bool sym_taps = false;                     // PFB kernel taps exactly symmetric (Tk == T)
    int phase_R = 1;                           // oversampled N = 4096 PFB: hop = N / phase_R, run as
                                               // phase_R critically sampled passes (see push_core)
    int16_t* d_view = nullptr;                 // phase passes: contiguous copy of [carry | buffer]
    int64_t view_cap = 0;                      //   when the push is not 16-byte aligned (samples)
    void* d_ptones = nullptr;                  // phase passes: each pass's tones [pass][tone][frame]
    int64_t ptones_cap = 0;                    //   frames per pass row
    void* d_pre = nullptr;                     // FIR pre-sum rows (rfr::pfb_pre_rows plans)
    int64_t pre_cap = 0;                       //   [frame][N] float2, frames
    bool gen = false;                          // PFB through the any-N kernels
    rfr::GenPlan gplan;
    int32_t L = 0, D = 0, Lpad = 0;            // demod
    int64_t W = 0, H = 0;                      // window and hop (samples)
    uint32_t out_flags = 0;
    rfr_window window{};
    std::vector<uint64_t> words;
    std::vector<int32_t> bins;
    std::vector<double> h64;                   // prototype, FP64 (length N*T or L)
    std::vector<float> h32;
    int device = 0, n_sms = 0, max_smem = 0;

    // device tables
    float* d_h = nullptr;          // PFB kernel taps [Tk*N] (zero-padded oldest taps)
    void* d_tw = nullptr;          // FFT twiddles
    void* d_tw_cl = nullptr;       // cluster PFB kernel's twiddles (N = 8192, 16384 with T <= 8)
    int tw_cl_count = 0;
    int tw_count = 0;
    int32_t* d_bins = nullptr;
    uint64_t* d_words = nullptr;
    uint64_t* d_rates = nullptr;   // chirp mode: rate words (d_words holds the start words)
    std::vector<uint64_t> rates;
    float* d_h32 = nullptr;        // taps as FP32 (plain forms)
    void* d_c32 = nullptr;         // plain demod: FP32 modulated taps [tones][L]
    void* d_bhi = nullptr;         // demod modulated taps, fp16 hi/lo
    void* d_blo = nullptr;
    int32_t ntp = 0;               // demod tones padded
    int tap_exp = 0;               // demod power-of-two tap scale exponent
    int accum_chunk = 2;           // demod: K blocks per TMEM accumulation chunk
    int demod_products = 4;        // demod GEMM form: 4 (real embedding) or 3 (Gauss)
    void* d_b3 = nullptr;          // three-product form: six tap planes
    void* d_xs3 = nullptr;         // three-product form: six source planes
    int64_t xs3_rows_cap = 0;
    int32_t Lpad3 = 0, ntp3 = 0, tap_exp3 = 0;
    int* d_status = nullptr;

    // stream state
    int64_t samples = 0;           // samples consumed
    int64_t frames = 0;            // frames produced
    int64_t cl = 0;                // carry length (may be <= 0: samples to skip)
    int16_t* d_carry[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t carry_cap = 0;

    // demod scratch
    void* d_xs_hi = nullptr;
    void* d_xs_lo = nullptr;
    int64_t xs_rows_cap = 0;
    void* d_rot = nullptr;
    int64_t rot_cap = 0;

    // queued output ring (rfr_push / rfr_pull)
    void* d_qfull = nullptr;
    void* d_qtones = nullptr;
    int64_t q_cap = 0;             // frames
    int64_t q_frames = 0;          // pending frames
    cudaStream_t last_stream = nullptr;

    // host-staging (rfr_process_host)
    static constexpr int kStageBufs = 3;       // chunks in flight (copy in, compute, copy out)
    void* d_stage_in[kStageBufs] = {};
    void* d_stage_full[kStageBufs] = {};
    int64_t stage_samples = 0;
    cudaStream_t stage_st[kStageBufs] = {};
    cudaEvent_t stage_ev[kStageBufs] = {};
    // tone rows leave the device in groups of chunks (long rows for the
    // strided device-to-host copy); two group buffers alternate
    static constexpr int kToneGroups = 2;
    void* d_tgroup[kToneGroups] = {};
    int64_t tgroup_cap = 0;        // frames per row of a group buffer
    cudaEvent_t tgroup_ev[kToneGroups] = {};

    // plain-form scratch
    void* plain_scratch = nullptr;
    size_t plain_scratch_bytes = 0;
    void* plain_fft = nullptr;
    int64_t plain_fft_batch = 0;
    void* plain_blas = nullptr;    // cuBLAS handle of the Cgemm form

    rfr::TuneConfig tune;
    std::string last_error;
};

namespace rfr {
// Enqueue one push of [carry | iq] into `o` on `st` (no allocation when the
// scratch is already large enough; see ensure_scratch).
rfr_status push_core(rfr_plan* p, const int16_t* iq, int64_t n, const rfr_output* o,
                     int64_t* frames_out, cudaStream_t st, DemodGemmJob* defer_gemm = nullptr);
// Grow the plan's per-push scratch for a push of n samples (may allocate and
// synchronise the device; never call it during stream capture).
rfr_status ensure_scratch(rfr_plan* p, int64_t n);
int64_t frames_for_samples(const rfr_plan* p, int64_t n);
// Argument and capacity checks of push_core without side effects.
rfr_status push_check(rfr_plan* p, const int16_t* iq, int64_t n, const rfr_output* o);
}  // namespace rfr
