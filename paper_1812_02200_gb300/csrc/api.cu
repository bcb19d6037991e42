// api.cu -- the C ABI (include/rfr.h): plan creation, streaming pushes,
// queued pull, host-staged processing, checkpoint/resume and the plain FP32
// comparison entry point.  All device work is enqueued on the caller's stream;
// the stream state (carry of history + residue, position) stays on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "dev_common.cuh"
#include "fft_dev.cuh"
#include "rfr_internal.h"
#include "trace.h"

using rfr::DEV_OK;
using rfr::DEV_TIMEOUT;

namespace {

constexpr double kPi = 3.14159265358979323846;

rfr_status fail(rfr_plan* p, rfr_status st, const char* msg) {
    if (p) p->last_error = msg;
    return st;
}

rfr_status cuda_fail(rfr_plan* p, cudaError_t e, const char* where) {
    if (p) {
        p->last_error = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return e == cudaErrorMemoryAllocation ? RFR_E_NOMEM : RFR_E_CUDA;
}

#define RFR_CUDA(p, call)                                      \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail((p), e_, #call); \
    } while (0)

template <typename T>
cudaError_t dev_alloc(T** ptr, size_t bytes) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, bytes ? bytes : 16);
    *ptr = static_cast<T*>(v);
    return e;
}

void dev_free(void* p) {
    if (p) cudaFree(p);
}

// FFT twiddle tables for an N-point frame (layout of fft_dev.cuh), FP64 -> FP32.
std::vector<float> make_twiddles(int log2n) {
    std::vector<float> t;
    const int n = 1 << log2n;
    const int p16 = log2n / 4, rf = 1 << (log2n % 4);
    auto push = [&](int64_t num, int64_t den) {
        const double a = -2.0 * kPi * static_cast<double>(num) / static_cast<double>(den);
        t.push_back(static_cast<float>(std::cos(a)));
        t.push_back(static_cast<float>(std::sin(a)));
    };
    int ns = 16;
    for (int s = 1; s < p16; ++s, ns *= 16)
        for (int r = 1; r < 16; ++r)
            for (int k = 0; k < ns; ++k) push(static_cast<int64_t>(r) * k, 16LL * ns);
    if (rf > 1) {
        const int span = n / rf;
        for (int r = 1; r < rf; ++r)
            for (int j = 0; j < span; ++j) push(static_cast<int64_t>(r) * j, n);
    }
    return t;
}

// ------------------------------------------------- phase-pass tone rows
// Output frame f = R m + k of tone t comes from column m of pass k's dense
// row.  Grid rows are tones; a thread takes column m of the R pass rows
// (coalesced loads across the warp) and writes output frames R m .. R m + R - 1.
__global__ void interleave_tones_kernel(const float2* __restrict__ src, int64_t src_ld, int R, int n_tones,
                                        int64_t F, float2* __restrict__ out, int64_t ld) {
    const int64_t M = (F + R - 1) / R;
    const int64_t pass = static_cast<int64_t>(n_tones) * src_ld;
    for (int t = blockIdx.y; t < n_tones; t += gridDim.y) {
        const float2* s = src + static_cast<int64_t>(t) * src_ld;
        float2* o = out + static_cast<int64_t>(t) * ld;
        for (int64_t m = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; m < M;
             m += static_cast<int64_t>(gridDim.x) * blockDim.x) {
            float2 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < R) v[k] = s[k * pass + m];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < R && m * R + k < F) o[m * R + k] = v[k];
        }
    }
}

// -------------------------------------------------------------- carry copy
__global__ void carry_update_kernel(const uint32_t* __restrict__ old_carry, int64_t cl,
                                    const uint32_t* __restrict__ buf, int64_t from, int64_t count,
                                    uint32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t idx = from + i;
        out[i] = idx < cl ? old_carry[idx] : buf[idx - cl];
    }
}

// Self-test of the bounded waits: one thread waits on an mbarrier phase that
// nothing completes; the wait must give up after limit_ns and record
// DEV_TIMEOUT (no trap, no fault).
__global__ void wait_selftest_kernel(int* status, uint64_t limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        rfr::mbar_init(&bar, 1);
        rfr::fence_mbar_init();
        rfr::mbar_wait(&bar, 0, status, limit_ns);   // phase 0 never completes
    }
}

int64_t frames_for_len(const rfr_plan* p, int64_t lv) {
    return lv >= p->W ? (lv - p->W) / p->H + 1 : 0;
}

bool out_ok(const rfr_plan* p, const rfr_output* o, int64_t F) {
    if (F == 0) return true;
    if (o->frame_offset < 0) return false;
    if (p->mode == RFR_MODE_PFB && (p->out_flags & RFR_OUT_FULL)) {
        if (!o->full || o->full_ld < p->N || o->full_cap < o->frame_offset + F) return false;
    }
    const bool want_tones = p->mode != RFR_MODE_PFB || (p->out_flags & RFR_OUT_TONES);
    if (want_tones && !p->words.empty()) {
        if (!o->tones || o->tones_cap < o->frame_offset + F || o->tones_ld < o->frame_offset + F)
            return false;
    }
    return true;
}

rfr_status check_status(rfr_plan* p) {
    int st = 0;
    RFR_CUDA(p, cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st == DEV_TIMEOUT) return fail(p, RFR_E_TIMEOUT, "a device-side wait timed out");
    if (st != DEV_OK) return fail(p, RFR_E_CUDA, "device status error");
    return RFR_OK;
}

// RFR_DEBUG: wait for the call's work and report its errors at the call.
rfr_status debug_check(rfr_plan* p, cudaStream_t st, const char* what) {
    if (!rfr::debug_sync_allowed(st)) return RFR_OK;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(p, e, what);
    return check_status(p);
}

// Growth synchronises the device and allocates, which a stream capture
// cannot contain: refused (RFR_E_INVALID) while `st` is being captured.
rfr_status refuse_growth_in_capture(rfr_plan* p, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    RFR_CUDA(p, cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)
        return fail(p, RFR_E_INVALID,
                    "demodulation scratch must grow for this push size: push once outside stream capture first");
    return RFR_OK;
}

// F0 < 0: size the rotation table for the worst alignment of the first frame.
// st: the stream of the push that needs the scratch (checked for capture).
rfr_status ensure_demod_scratch(rfr_plan* p, int64_t F, int64_t F0, cudaStream_t st) {
    {
        const int64_t rows3 = p->demod_products == 3
                                  ? static_cast<int64_t>(rfr::demod3_xs_rows(F, p->Lpad3, p->D)) : 0;
        const int64_t rows = p->demod_products == 3 ? 0 : static_cast<int64_t>(rfr::demod_xs_rows(F, p->Lpad, p->D));
        const int64_t ntp = p->demod_products == 3 ? p->ntp3 : p->ntp;
        const int64_t anchors = F0 >= 0 ? rfr::demod_anchor_rows(F0, F) : (F + rfr::kDemodBM - 2) / rfr::kDemodBM + 1;
        const int64_t rot = anchors * ntp + ntp * rfr::kDemodBM;
        if (rows3 > p->xs3_rows_cap || rows > p->xs_rows_cap || rot > p->rot_cap) {
            const rfr_status rs = refuse_growth_in_capture(p, st);
            if (rs != RFR_OK) return rs;
        }
    }
    if (p->demod_products == 3) {
        // six fp16 planes [rows][D] of the Gauss three-product form
        const int64_t rows3 = static_cast<int64_t>(rfr::demod3_xs_rows(F, p->Lpad3, p->D));
        if (rows3 > p->xs3_rows_cap) {
            cudaDeviceSynchronize();
            dev_free(p->d_xs3);
            p->d_xs3 = nullptr;
            p->xs3_rows_cap = 0;
            RFR_CUDA(p, dev_alloc(&p->d_xs3, static_cast<size_t>(rows3) * 6 * p->D * sizeof(uint16_t)));
            p->xs3_rows_cap = rows3;
        }
    }
    const int64_t rows = p->demod_products == 3 ? 0 : static_cast<int64_t>(rfr::demod_xs_rows(F, p->Lpad, p->D));
    if (rows > p->xs_rows_cap) {
        cudaDeviceSynchronize();
        dev_free(p->d_xs_hi);
        dev_free(p->d_xs_lo);
        p->d_xs_hi = p->d_xs_lo = nullptr;
        p->xs_rows_cap = 0;
        const size_t bytes = static_cast<size_t>(rows) * 2 * p->D * sizeof(uint16_t);
        RFR_CUDA(p, dev_alloc(&p->d_xs_hi, bytes));
        RFR_CUDA(p, dev_alloc(&p->d_xs_lo, bytes));
        p->xs_rows_cap = rows;
    }
    const int64_t ntp = p->demod_products == 3 ? p->ntp3 : p->ntp;
    const int64_t anchors = F0 >= 0 ? rfr::demod_anchor_rows(F0, F) : (F + rfr::kDemodBM - 2) / rfr::kDemodBM + 1;
    const int64_t rot = anchors * ntp + ntp * rfr::kDemodBM;
    if (rot > p->rot_cap) {
        cudaDeviceSynchronize();
        dev_free(p->d_rot);
        p->d_rot = nullptr;
        p->rot_cap = 0;
        RFR_CUDA(p, dev_alloc(&p->d_rot, static_cast<size_t>(rot) * 8));
        p->rot_cap = rot;
    }
    return RFR_OK;
}

// Oversampled N = 4096 PFB as phase passes.  With hop H = N/R, frame
// j = R*i + k of the push starts at view sample i*N + k*H, so the frames of
// phase k are the critically sampled PFB of the view shifted by k*H samples
// (one fused-kernel launch), written to full rows fo + k + R*i (row pitch
// R*ld) and tone columns fo + k + R*i (column stride R).  The channel phase
// of the absolute time origin is exp(-2*pi*i*c*s/N) with s = (a0 + k*H) mod N
// a multiple of H, i.e. (-i)^(c*m) with m = s/H (R = 4) or (-1)^(c*m)
// (R = 2): an exact swap/negation of each bin, applied by the kernel.  A
// push that is not 16-byte aligned (or whose carry is not a multiple of 4
// samples) first copies [carry | buffer] into one aligned scratch view.
// Rows for the tones of every phase pass of a push of F frames: R x tones
// rows of ceil(F / R) frames, rounded up to an even count (the tone tile's
// TMA stores need 16-byte row pitches).  Grows outside stream capture only.
cudaError_t ensure_pass_tones(rfr_plan* p, int64_t F, cudaStream_t st) {
    const int nt = static_cast<int>(p->words.size());
    if (nt == 0 || !(p->out_flags & RFR_OUT_TONES)) return cudaSuccess;
    const int64_t need = ((F + p->phase_R - 1) / p->phase_R + 1) & ~int64_t(1);
    if (need <= p->ptones_cap) return cudaSuccess;
    if (st) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        if (cs != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
    }
    cudaDeviceSynchronize();
    dev_free(p->d_ptones);
    p->d_ptones = nullptr;
    p->ptones_cap = 0;
    const cudaError_t e = dev_alloc(&p->d_ptones, static_cast<size_t>(p->phase_R) * nt * need * 8);
    if (e == cudaSuccess) p->ptones_cap = need;
    return e;
}

rfr_status phase_passes(rfr_plan* p, const rfr::PfbLaunch& L0, const rfr_output* o, int64_t lv, int64_t F,
                        cudaStream_t st) {
    const int R = p->phase_R;
    const int64_t H = p->H, N = p->N;
    const int16_t* vcarry = L0.carry;
    const int16_t* vbuf = L0.buf;
    int64_t vcl = L0.cl;
    const bool aligned = (reinterpret_cast<uintptr_t>(L0.buf) % 16 == 0) && (L0.cl % 4 == 0) &&
                         (reinterpret_cast<uintptr_t>(L0.carry) % 16 == 0);
    if (!aligned) {
        if (lv > p->view_cap) {
            const rfr_status rs = refuse_growth_in_capture(p, st);
            if (rs != RFR_OK) return rs;
            cudaDeviceSynchronize();
            dev_free(p->d_view);
            p->d_view = nullptr;
            p->view_cap = 0;
            RFR_CUDA(p, dev_alloc(&p->d_view, static_cast<size_t>(lv) * 4));
            p->view_cap = lv;
        }
        RFR_CUDA(p, rfr::carry_update(L0.carry, L0.cl, L0.buf, L0.n, 0, lv, p->d_view, st));
        vcarry = p->d_view;
        vbuf = p->d_view;
        vcl = 0;
    }
    // each pass writes its tones as dense rows [k][tone][i] through the tone
    // tile's TMA stores; one kernel then interleaves them into [tone][frame]
    // (written at a column stride of R, each 32-byte sector of a tone row
    // would be filled by R launches, partially each time)
    const int nt = static_cast<int>(p->words.size());
    if (L0.tones) {
        const cudaError_t e = ensure_pass_tones(p, F, st);
        if (e == cudaErrorStreamCaptureUnsupported)
            return fail(p, RFR_E_INVALID, "push inside stream capture would grow the plan's scratch; push that size once before capturing");
        RFR_CUDA(p, e);
    }
    for (int k = 0; k < R; ++k) {
        const int64_t Fk = (F - k + R - 1) / R;           // frames R*i + k < F
        if (Fk <= 0) continue;
        const int64_t off = k * H;
        rfr::PfbLaunch L = L0;
        if (off < vcl) {
            L.carry = vcarry + 2 * off;
            L.cl = vcl - off;
            L.buf = vbuf;
        } else {
            L.carry = vcarry;
            L.cl = 0;
            L.buf = vbuf + 2 * (off - vcl);
        }
        L.n = (lv - off) - L.cl;
        L.F = Fk;
        L.frame_offset = 0;
        L.hop = static_cast<int>(N);
        if (L0.full) {
            L.full = static_cast<float2*>(L0.full) + (o->frame_offset + k) * o->full_ld;
            L.full_ld = R * o->full_ld;
        }
        if (L0.tones) {
            L.tones = static_cast<float2*>(p->d_ptones) + static_cast<int64_t>(k) * nt * p->ptones_cap;
            L.tones_ld = p->ptones_cap;
            L.tone_cs = 1;
        }
        const int64_t s = ((L0.a0 + off) % N + N) % N;     // a multiple of H
        const int m = static_cast<int>(s / H);
        L.rot = R == 4 ? m : 2 * m;
        L.a0 = L0.a0 + off;
        RFR_CUDA(p, rfr::pfb_launch(L, st));
    }
    if (L0.tones)
        RFR_CUDA(p, rfr::interleave_tones(p->d_ptones, p->ptones_cap, R, nt, F,
                                          static_cast<float2*>(L0.tones) + o->frame_offset, o->tones_ld, st));
    return RFR_OK;
}

}  // namespace

namespace rfr {
int64_t frames_for_samples(const rfr_plan* p, int64_t n) { return frames_for_len(p, p->cl + n); }

rfr_status push_check(rfr_plan* p, const int16_t* iq, int64_t n, const rfr_output* o) {
    if (n < 0 || (n > 0 && iq == nullptr)) return fail(p, RFR_E_INVALID, "bad input buffer");
    if (!out_ok(p, o, frames_for_len(p, p->cl + n))) return fail(p, RFR_E_SHORT, "output buffers missing or too small");
    return RFR_OK;
}

// The FIR pre-sum rows of F frames (PFB plans with rfr::pfb_pre_rows);
// growing them is refused while `st` is being captured (st null: not
// capturing).
rfr_status ensure_pre_rows(rfr_plan* p, int64_t F, cudaStream_t st) {
    if (F <= p->pre_cap) return RFR_OK;
    if (st) {
        const rfr_status rs = refuse_growth_in_capture(p, st);
        if (rs != RFR_OK) return rs;
    }
    cudaDeviceSynchronize();
    dev_free(p->d_pre);
    p->d_pre = nullptr;
    p->pre_cap = 0;
    RFR_CUDA(p, dev_alloc(&p->d_pre, static_cast<size_t>(F) * p->N * 8));
    p->pre_cap = F;
    return RFR_OK;
}

rfr_status ensure_scratch(rfr_plan* p, int64_t n) {
    // the most frames a push of n samples can complete whatever the stream's
    // state (a carried residue adds up to hop - 1 samples: the carry holds at
    // most W - 1), with the rotation table sized for any first frame, so that
    // later pushes of up to n samples never allocate (nor synchronise)
    const int64_t F = frames_for_len(p, std::max<int64_t>(p->cl, p->W - 1) + n);
    if (p->mode == RFR_MODE_PFB && p->gen && F > 0) RFR_CUDA(p, rfr::gen_plan_reserve(&p->gplan, F));
    if (p->mode == RFR_MODE_PFB && (p->phase_R > 1 || (!p->gen && rfr::pfb_split16(p->log2n, p->Tk)))) {
        const int64_t lv = std::max<int64_t>(p->cl, p->W - 1) + n;
        if (lv > p->view_cap) {
            cudaDeviceSynchronize();
            dev_free(p->d_view);
            p->d_view = nullptr;
            p->view_cap = 0;
            RFR_CUDA(p, dev_alloc(&p->d_view, static_cast<size_t>(lv) * 4));
            p->view_cap = lv;
        }
        if (p->phase_R > 1) RFR_CUDA(p, ensure_pass_tones(p, F, nullptr));
    }
    if (p->mode == RFR_MODE_PFB && !p->gen && p->phase_R == 1 && rfr::pfb_pre_rows(p->log2n, p->Tk)) {
        const rfr_status rs = ensure_pre_rows(p, F, nullptr);
        if (rs != RFR_OK) return rs;
    }
    if (p->mode == RFR_MODE_DEMOD && F > 0 && !p->words.empty()) return ensure_demod_scratch(p, F, -1, nullptr);
    return RFR_OK;
}

// Core of every push: enqueue the frames of [carry | buf] into `out`.
// defer_gemm (batched steps): a three-product demodulation plan leaves its
// GEMM to the caller's persistent launch, described in *defer_gemm
// (n_tiles = 0 when the plan has nothing to launch or is another form).
rfr_status push_core(rfr_plan* p, const int16_t* iq, int64_t n, const rfr_output* o,
                     int64_t* frames_out, cudaStream_t st, rfr::DemodGemmJob* defer_gemm) {
    if (defer_gemm) defer_gemm->n_tiles = 0;
    if (n < 0 || (n > 0 && iq == nullptr)) return fail(p, RFR_E_INVALID, "bad input buffer");
    const int64_t lv = p->cl + n;
    const int64_t F = frames_for_len(p, lv);
    if (!out_ok(p, o, F)) return fail(p, RFR_E_SHORT, "output buffers missing or too small");
    const int16_t* carry = p->d_carry[p->cur];
    if (F > 0) {
        if (p->mode == RFR_MODE_PFB) {
            rfr::PfbLaunch L{};
            L.carry = carry;
            L.cl = p->cl;
            L.buf = iq;
            L.n = n;
            L.F = F;
            L.log2n = p->log2n;
            L.taps_kernel = p->Tk;
            L.h = p->d_h;
            L.tw = p->d_tw;
            L.tw_count = p->tw_count;
            L.bins = p->d_bins;
            L.n_tones = (p->out_flags & RFR_OUT_TONES) ? static_cast<int>(p->words.size()) : 0;
            L.full = (p->out_flags & RFR_OUT_FULL) ? o->full : nullptr;
            L.full_ld = o->full_ld;
            L.tones = o->tones;
            L.tones_ld = o->tones_ld;
            L.frame_offset = o->frame_offset;
            L.status = p->d_status;
            L.n_sms = p->n_sms;
            L.max_smem = p->max_smem;
            L.lookahead = p->tune.pfb_lookahead;
            L.hop = static_cast<int>(p->H);
            L.a0 = p->samples - p->cl;
            L.sym_taps = p->sym_taps ? 1 : 0;
            L.cluster = p->tune.pfb_cluster && p->d_tw_cl ? 1 : 0;
            L.tw_cl = p->d_tw_cl;
            L.tw_cl_count = p->tw_cl_count;
            if (p->gen && p->gplan.N1 > 1 && p->gplan.z_frames < std::min(F, p->gplan.z_cap_frames)) {
                // grow the between-pass buffer, unless the stream is being
                // captured (then the frames go through the buffer in batches)
                cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
                RFR_CUDA(p, cudaStreamIsCapturing(st, &cs));
                if (cs == cudaStreamCaptureStatusNone) RFR_CUDA(p, rfr::gen_plan_reserve(&p->gplan, F));
                else if (p->gplan.z_frames < 1)
                    return fail(p, RFR_E_INVALID, "reserve scratch (a push outside capture) before capturing");
            }
            if (p->phase_R > 1) {
                rfr_status rs = phase_passes(p, L, o, lv, F, st);
                if (rs != RFR_OK) return rs;
            } else if (!p->gen && rfr::pfb_split16(p->log2n, p->Tk)) {
                // the two-pass 16-tap form needs a 16-byte aligned view: an
                // unaligned push goes through a contiguous copy of it.  Scratch
                // that has to grow is sized for a push of n samples after any
                // carry (so that a later push of that size never grows it)
                const int64_t lv_max = std::max<int64_t>(p->cl, p->W - 1) + n;
                const bool aligned = (reinterpret_cast<uintptr_t>(iq) % 16 == 0) && (p->cl % 4 == 0) &&
                                     (reinterpret_cast<uintptr_t>(carry) % 16 == 0);
                if (!aligned) {
                    if (lv > p->view_cap) {
                        const rfr_status rs = refuse_growth_in_capture(p, st);
                        if (rs != RFR_OK) return rs;
                        cudaDeviceSynchronize();
                        dev_free(p->d_view);
                        p->d_view = nullptr;
                        p->view_cap = 0;
                        RFR_CUDA(p, dev_alloc(&p->d_view, static_cast<size_t>(lv_max) * 4));
                        p->view_cap = lv_max;
                    }
                    RFR_CUDA(p, rfr::carry_update(carry, p->cl, iq, n, 0, lv, p->d_view, st));
                    L.carry = p->d_view;
                    L.cl = 0;
                    L.buf = p->d_view;
                    L.n = lv;
                }
                const rfr_status rs = ensure_pre_rows(p, F <= p->pre_cap ? F : frames_for_len(p, lv_max), st);
                if (rs != RFR_OK) return rs;
                L.pre = p->d_pre;
                L.pre_cap = p->pre_cap;
                RFR_CUDA(p, rfr::pfb_launch(L, st));
            } else {
                if (!p->gen && rfr::pfb_pre_rows(p->log2n, p->Tk) && !L.cluster) {
                    // FIR pre-sum rows, sized for a push of n samples after any
                    // carry when they grow
                    const int64_t lv_max = std::max<int64_t>(p->cl, p->W - 1) + n;
                    const rfr_status rs = ensure_pre_rows(p, F <= p->pre_cap ? F : frames_for_len(p, lv_max), st);
                    if (rs != RFR_OK) return rs;
                    L.pre = p->d_pre;
                    L.pre_cap = p->pre_cap;
                }
                RFR_CUDA(p, p->gen ? rfr::gen_pfb_launch(L, p->gplan, st) : rfr::pfb_launch(L, st));
            }
        } else if (p->mode == RFR_MODE_CHIRP) {
            rfr::ChirpLaunch L{};
            L.carry = carry;
            L.cl = p->cl;
            L.buf = iq;
            L.F = F;
            L.a0 = p->samples - p->cl;
            L.L = p->L;
            L.D = p->D;
            L.h32 = p->d_h32;
            L.start_words = p->d_words;
            L.rate_words = p->d_rates;
            L.n_chirps = static_cast<int>(p->words.size());
            L.tones = o->tones;
            L.tones_ld = o->tones_ld;
            L.frame_offset = o->frame_offset;
            L.n_sms = p->n_sms;
            RFR_CUDA(p, rfr::chirp_demod_launch(L, st));
        } else {
            if (!p->words.empty()) {
                rfr_status rs = ensure_demod_scratch(p, F, p->frames, st);
                if (rs != RFR_OK) return rs;
                rfr::DemodLaunch L{};
                L.carry = carry;
                L.cl = p->cl;
                L.buf = iq;
                L.n = n;
                L.F = F;
                L.a0 = p->samples - p->cl;
                L.F0 = p->frames;
                L.L = p->L;
                L.D = p->D;
                L.Lpad = p->Lpad;
                L.n_tones = static_cast<int>(p->words.size());
                L.ntp = p->ntp;
                L.words = p->d_words;
                L.b_hi = p->d_bhi;
                L.b_lo = p->d_blo;
                L.inv_scale = std::ldexp(1.0, -p->tap_exp);
                L.xs_hi = p->d_xs_hi;
                L.xs_lo = p->d_xs_lo;
                L.xs_rows = p->xs_rows_cap;
                L.rot = p->d_rot;
                L.tones = o->tones;
                L.tones_ld = o->tones_ld;
                L.frame_offset = o->frame_offset;
                L.status = p->d_status;
                L.n_sms = p->n_sms;
                L.kchunk = p->accum_chunk;
                L.raster_group = p->tune.demod_raster;
                if (p->demod_products == 3) {
                    L.Lpad = p->Lpad3;
                    L.ntp = p->ntp3;
                    L.b_hi = p->d_b3;
                    L.b_lo = nullptr;
                    L.inv_scale = std::ldexp(1.0, -p->tap_exp3);
                    L.xs_hi = p->d_xs3;
                    L.xs_lo = nullptr;
                    L.xs_rows = p->xs3_rows_cap;
                    L.tone_tile = p->tune.demod_bt;
                    L.fused_presplit = p->tune.demod_fused;
                    L.pair = p->tune.demod_pair;
                    if (defer_gemm) RFR_CUDA(p, rfr::demod3_prepare(L, st, defer_gemm));
                    else RFR_CUDA(p, rfr::demod3_launch(L, st));
                } else {
                    RFR_CUDA(p, rfr::demod_launch(L, st));
                }
            }
        }
    }
    // new carry = v[F*H, lv)
    const int64_t ncl = lv - F * p->H;
    if (ncl > 0) {
        if (ncl > p->carry_cap) return fail(p, RFR_E_INVALID, "internal: carry overflow");
        RFR_CUDA(p, rfr::carry_update(carry, p->cl, iq, n, F * p->H, ncl, p->d_carry[p->cur ^ 1], st));
        p->cur ^= 1;
    }
    p->cl = ncl;
    p->samples += n;
    p->frames += F;
    p->last_stream = st;
    if (frames_out) *frames_out = F;
    return RFR_OK;
}
}  // namespace rfr

namespace {
using rfr::push_core;

rfr_status reset_state(rfr_plan* p) {
    p->samples = 0;
    p->frames = 0;
    p->q_frames = 0;
    p->cur = 0;
    p->cl = p->W - p->H;     // zero history (negative: samples skipped before frame 0)
    if (p->carry_cap > 0) {
        RFR_CUDA(p, cudaMemset(p->d_carry[0], 0, static_cast<size_t>(p->carry_cap) * 4));
        RFR_CUDA(p, cudaMemset(p->d_carry[1], 0, static_cast<size_t>(p->carry_cap) * 4));
    }
    RFR_CUDA(p, cudaMemset(p->d_status, 0, sizeof(int)));
    return RFR_OK;
}

void destroy(rfr_plan* p) {
    if (!p) return;
    cudaDeviceSynchronize();
    for (void* q : {static_cast<void*>(p->d_h), p->d_tw, p->d_tw_cl, static_cast<void*>(p->d_bins),
                    static_cast<void*>(p->d_words), static_cast<void*>(p->d_rates), static_cast<void*>(p->d_h32), p->d_c32, p->d_bhi, p->d_blo,
                    static_cast<void*>(p->d_status), static_cast<void*>(p->d_carry[0]),
                    static_cast<void*>(p->d_carry[1]), p->d_xs_hi, p->d_xs_lo, p->d_rot, p->d_qfull, p->d_b3, p->d_xs3,
                    p->d_qtones, static_cast<void*>(p->d_view), p->d_ptones, p->d_pre})
        dev_free(q);
    for (int i = 0; i < rfr_plan::kStageBufs; ++i) {
        dev_free(p->d_stage_in[i]);
        dev_free(p->d_stage_full[i]);
        if (p->stage_st[i]) cudaStreamDestroy(p->stage_st[i]);
    }
    for (auto& e : p->stage_ev)
        if (e) cudaEventDestroy(e);
    for (int g = 0; g < rfr_plan::kToneGroups; ++g) {
        dev_free(p->d_tgroup[g]);
        if (p->tgroup_ev[g]) cudaEventDestroy(p->tgroup_ev[g]);
    }
    rfr::plain_release(p->plain_scratch, p->plain_fft, p->plain_blas);
    rfr::gen_plan_free(&p->gplan);
    delete p;
}

}  // namespace

namespace rfr {
cudaError_t carry_update(const int16_t* old_carry, int64_t cl, const int16_t* buf, int64_t n,
                         int64_t from, int64_t count, int16_t* new_carry, cudaStream_t st) {
    (void)n;
    if (count <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((count + threads - 1) / threads, 4096);
    carry_update_kernel<<<static_cast<unsigned>(blocks), threads, 0, st>>>(
        reinterpret_cast<const uint32_t*>(old_carry), cl, reinterpret_cast<const uint32_t*>(buf),
        from, count, reinterpret_cast<uint32_t*>(new_carry));
    return cudaGetLastError();
}

cudaError_t interleave_tones(const void* src, int64_t src_ld, int R, int n_tones, int64_t F, void* out,
                             int64_t ld, cudaStream_t st) {
    if (F <= 0 || n_tones <= 0) return cudaSuccess;
    if (R < 1 || R > 4) return cudaErrorInvalidValue;
    const int64_t M = (F + R - 1) / R;
    const dim3 grid(static_cast<unsigned>(std::min<int64_t>((M + 255) / 256, 65535)),
                    static_cast<unsigned>(std::min(n_tones, 65535)));
    interleave_tones_kernel<<<grid, 256, 0, st>>>(static_cast<const float2*>(src), src_ld, R, n_tones, F,
                                                  static_cast<float2*>(out), ld);
    return cudaGetLastError();
}
}  // namespace rfr

// ===================================================================== ABI
extern "C" {

const char* rfr_version(void) { return "rfr 0.1 (sm_103a)"; }

const char* rfr_status_string(rfr_status s) {
    switch (s) {
    case RFR_OK: return "ok";
    case RFR_E_INVALID: return "invalid argument";
    case RFR_E_NOMEM: return "out of memory";
    case RFR_E_CUDA: return "CUDA error";
    case RFR_E_TIMEOUT: return "device wait timed out";
    case RFR_E_SHORT: return "output capacity too small";
    case RFR_E_BUSY: return "busy";
    case RFR_E_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* rfr_last_error(const rfr_plan* p) { return p ? p->last_error.c_str() : ""; }

uint64_t rfr_freq_to_word(double f_hz, double fs_hz) { return rfr::freq_to_word(f_hz, fs_hz); }

int32_t rfr_word_to_bin(uint64_t word, int32_t n) { return rfr::word_to_bin(word, n); }

rfr_status rfr_plan_create(rfr_plan** out, int32_t channels, int32_t taps, const rfr_window* window,
                           const rfr_tones* tones, int32_t decimation, uint32_t out_flags) {
    if (!out || !window) return RFR_E_INVALID;
    *out = nullptr;
    if (window->kind < RFR_WIN_RECT || window->kind > RFR_WIN_KAISER) return RFR_E_INVALID;
    if (!(window->cutoff >= 0.0) || !(window->cutoff < 0.5) || !std::isfinite(window->beta))
        return RFR_E_INVALID;
    const int32_t nt = tones ? tones->count : 0;
    if (nt < 0 || nt > 65536 || (nt > 0 && !tones->words)) return RFR_E_INVALID;

    rfr_plan* p = new (std::nothrow) rfr_plan();
    if (!p) return RFR_E_NOMEM;
    p->window = *window;
    p->out_flags = out_flags;
    if (nt > 0) p->words.assign(tones->words, tones->words + nt);
    cudaGetDevice(&p->device);
    cudaDeviceGetAttribute(&p->n_sms, cudaDevAttrMultiProcessorCount, p->device);
    cudaDeviceGetAttribute(&p->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);

    auto bad = [&](rfr_status s) {
        destroy(p);
        return s;
    };

    if (channels > 0) {
        // ------------------------------------------------------------- PFB
        if (channels < 2 || channels > (1 << 24)) return bad(RFR_E_INVALID);
        if (taps < 1 || taps > 16 || decimation < 1 || decimation > channels) return bad(RFR_E_INVALID);
        if (out_flags == 0 || (out_flags & ~uint32_t(RFR_OUT_FULL | RFR_OUT_TONES)) != 0) return bad(RFR_E_INVALID);
        if ((out_flags & RFR_OUT_TONES) && nt == 0) return bad(RFR_E_INVALID);
        const bool pow2 = (channels & (channels - 1)) == 0;
        p->mode = RFR_MODE_PFB;
        p->N = channels;
        p->T = taps;
        // powers of two from 16 to 16384, critically sampled: the fused
        // single-CTA kernels; every other N = 2^a 3^b 5^c 7^d up to 2^24 and
        // every hop < N (oversampled): the mixed-radix kernels
        // N = 4096, T = 8 with hop N/2 or N/4: the oversampled frames are
        // N/hop interleaved critically sampled PFBs of the stream shifted by
        // k*hop (k < N/hop), each rotated by an exact quarter-turn power per
        // bin (the channel phase of the absolute time origin), so they run on
        // the symmetric-tap fused kernel as phase passes
        const bool phase = pow2 && channels == 4096 && taps == 8 && (decimation == 2048 || decimation == 1024);
        p->gen = !phase && (!pow2 || channels < 16 || channels > 16384 || decimation != channels);
        p->phase_R = phase ? channels / decimation : 1;
        if (p->gen && !rfr::gen_supported(channels)) return bad(RFR_E_UNSUPPORTED);
        if (p->gen) {
            p->Tk = taps;
        } else {
            while ((1 << p->log2n) < channels) ++p->log2n;
            p->Tk = rfr::pfb_kernel_taps(p->log2n, taps);
        }
        const int64_t M = static_cast<int64_t>(channels) * taps;
        p->h64.resize(M);
        const double fc = window->cutoff > 0.0 ? window->cutoff : 0.5 / channels;
        if (rfr::build_lowpass(window->kind, window->beta, fc, M, p->h64.data()) != 0) return bad(RFR_E_INVALID);
        // FP32 taps, exactly symmetric like the prototype itself (its FP64
        // evaluation can differ in the last bit between h[j] and h[M-1-j]):
        // the rounding of the mean of the two, within one FP32 ulp of either
        p->h32.resize(M);
        for (int64_t j = 0; j < M; ++j) p->h32[j] = static_cast<float>(0.5 * (p->h64[j] + p->h64[M - 1 - j]));
        p->sym_taps = p->Tk == taps;
        // kernel taps: zero-padded at the oldest end to Tk*N
        std::vector<float> hk(static_cast<size_t>(p->Tk) * channels, 0.0f);
        std::copy(p->h32.begin(), p->h32.end(), hk.begin() + static_cast<size_t>(p->Tk - taps) * channels);
        p->bins.resize(nt);
        for (int s = 0; s < nt; ++s) p->bins[s] = rfr::word_to_bin(p->words[s], channels);
        std::vector<float> tw = p->gen ? std::vector<float>() : make_twiddles(p->log2n);
        p->tw_count = static_cast<int>(tw.size() / 2);
        std::vector<float> tw_cl;
        const int ccl = p->gen ? 0 : rfr::pfb_cluster_size(p->log2n, p->Tk);
        if (ccl > 0) {
            // the cluster kernel's table: the 4096-point FFT's twiddles, then
            // W_N^(k2 p1) for k2 < C, p1 < 4096 (its cross-CTA step; FP64 -> FP32)
            tw_cl = make_twiddles(12);
            p->tw_cl_count = static_cast<int>(tw_cl.size() / 2);
            for (int k2 = 0; k2 < ccl; ++k2)
                for (int p1 = 0; p1 < 4096; ++p1) {
                    const double ang = -2.0 * kPi * static_cast<double>(k2 * p1) / static_cast<double>(channels);
                    tw_cl.push_back(static_cast<float>(std::cos(ang)));
                    tw_cl.push_back(static_cast<float>(std::sin(ang)));
                }
        }
        p->W = static_cast<int64_t>(p->Tk) * channels;
        p->H = decimation;
        p->carry_cap = p->W;
        cudaError_t e = cudaSuccess;
        if ((e = dev_alloc(&p->d_h, hk.size() * 4)) != cudaSuccess ||
            (e = dev_alloc(&p->d_h32, p->h32.size() * 4)) != cudaSuccess ||
            (e = dev_alloc(&p->d_tw, std::max<size_t>(tw.size(), 2) * 4)) != cudaSuccess ||
            (e = dev_alloc(&p->d_bins, std::max<size_t>(nt, 1) * 4)) != cudaSuccess)
            return bad(cuda_fail(p, e, "plan alloc"));
        // the between-pass buffer of the two-pass form: 1 GB of frames (at
        // least one); large batches keep the launches few and their tails
        // short, which costs more here than Z's round trip through HBM
        if (p->gen && ((e = rfr::gen_plan_init(&p->gplan, channels, int64_t(1024) << 20)) != cudaSuccess ||
                       (e = rfr::gen_plan_set_tones(&p->gplan, p->bins.data(), nt)) != cudaSuccess))
            return bad(cuda_fail(p, e, "plan alloc"));
        cudaMemcpy(p->d_h, hk.data(), hk.size() * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(p->d_h32, p->h32.data(), p->h32.size() * 4, cudaMemcpyHostToDevice);
        if (!tw.empty()) cudaMemcpy(p->d_tw, tw.data(), tw.size() * 4, cudaMemcpyHostToDevice);
        if (!tw_cl.empty()) {
            if ((e = dev_alloc(&p->d_tw_cl, tw_cl.size() * 4)) != cudaSuccess) return bad(cuda_fail(p, e, "plan alloc"));
            cudaMemcpy(p->d_tw_cl, tw_cl.data(), tw_cl.size() * 4, cudaMemcpyHostToDevice);
        }
        if (nt) cudaMemcpy(p->d_bins, p->bins.data(), nt * 4, cudaMemcpyHostToDevice);
    } else if (channels == 0) {
        // ----------------------------------------------------------- demod
        if (taps < 1 || taps > 16384 || decimation < 32 || decimation % 32 != 0 ||
            decimation > (1 << 20))
            return bad(RFR_E_INVALID);
        if (out_flags != RFR_OUT_TONES) return bad(RFR_E_INVALID);
        p->mode = RFR_MODE_DEMOD;
        p->L = taps;
        p->D = decimation;
        p->Lpad = (taps + 31) / 32 * 32;
        p->h64.resize(taps);
        if (rfr::build_lowpass(window->kind, window->beta, window->cutoff, taps, p->h64.data()) != 0)
            return bad(RFR_E_INVALID);
        p->h32.resize(taps);
        for (int j = 0; j < taps; ++j) p->h32[j] = static_cast<float>(p->h64[j]);
        p->W = taps;
        p->H = decimation;
        p->carry_cap = std::max<int64_t>(taps, 1);
        p->ntp = (nt + rfr::kDemodBN / 2 - 1) / (rfr::kDemodBN / 2) * (rfr::kDemodBN / 2);
        double hmax = 0.0;
        for (double v : p->h64) hmax = std::max(hmax, std::fabs(v));
        int e2 = 0;
        std::frexp(hmax, &e2);               // hmax in [2^(e2-1), 2^e2)
        p->tap_exp = 15 - e2;                // hmax * 2^e in [2^14, 2^15)
        cudaError_t e = cudaSuccess;
        double* d_h64 = nullptr;
        if ((e = dev_alloc(&p->d_words, std::max<size_t>(nt, 1) * 8)) != cudaSuccess ||
            (e = dev_alloc(&p->d_h32, static_cast<size_t>(taps) * 4)) != cudaSuccess)
            return bad(cuda_fail(p, e, "plan alloc"));
        cudaMemcpy(p->d_h32, p->h32.data(), static_cast<size_t>(taps) * 4, cudaMemcpyHostToDevice);
        if (nt) {
            cudaMemcpy(p->d_words, p->words.data(), static_cast<size_t>(nt) * 8, cudaMemcpyHostToDevice);
            const size_t bbytes = static_cast<size_t>(2) * p->ntp * 2 * p->Lpad * sizeof(uint16_t);
            if ((e = dev_alloc(&p->d_bhi, bbytes)) != cudaSuccess ||
                (e = dev_alloc(&p->d_blo, bbytes)) != cudaSuccess ||
                (e = dev_alloc(&d_h64, static_cast<size_t>(taps) * 8)) != cudaSuccess) {
                dev_free(d_h64);
                return bad(cuda_fail(p, e, "plan alloc"));
            }
            cudaMemcpy(d_h64, p->h64.data(), static_cast<size_t>(taps) * 8, cudaMemcpyHostToDevice);
            e = rfr::demod_build_taps(d_h64, p->d_words, nt, p->ntp, taps, p->Lpad, p->tap_exp,
                                      p->d_bhi, p->d_blo, nullptr);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            dev_free(d_h64);
            if (e != cudaSuccess) return bad(cuda_fail(p, e, "modulated-tap build"));
        }
    } else {
        return bad(RFR_E_INVALID);
    }
    cudaError_t e = cudaSuccess;
    if ((e = dev_alloc(&p->d_status, sizeof(int))) != cudaSuccess ||
        (e = dev_alloc(&p->d_carry[0], static_cast<size_t>(p->carry_cap) * 4)) != cudaSuccess ||
        (e = dev_alloc(&p->d_carry[1], static_cast<size_t>(p->carry_cap) * 4)) != cudaSuccess)
        return bad(cuda_fail(p, e, "plan alloc"));
    if (reset_state(p) != RFR_OK) return bad(RFR_E_CUDA);
    // demodulation: the Gauss three-product form wherever D allows it
    if (p->mode == RFR_MODE_DEMOD && !p->words.empty() && p->D % 64 == 0 &&
        rfr_plan_set_demod_products(p, 3) != RFR_OK)
        return bad(RFR_E_CUDA);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bad(cuda_fail(p, e, "plan create"));
    *out = p;
    return RFR_OK;
}

rfr_status rfr_plan_create_chirp(rfr_plan** out, int32_t taps, const rfr_window* window,
                                 const uint64_t* start_words, const uint64_t* rate_words, int32_t n_chirps,
                                 int32_t decimation) {
    if (!out || !window || !start_words || !rate_words) return RFR_E_INVALID;
    *out = nullptr;
    if (window->kind < RFR_WIN_RECT || window->kind > RFR_WIN_KAISER || !(window->cutoff >= 0.0) ||
        !(window->cutoff < 0.5) || !std::isfinite(window->beta))
        return RFR_E_INVALID;
    if (taps < 1 || taps > 16384 || decimation < 1 || decimation > (1 << 24) || n_chirps < 1 || n_chirps > 4096)
        return RFR_E_INVALID;
    rfr_plan* p = new (std::nothrow) rfr_plan();
    if (!p) return RFR_E_NOMEM;
    p->mode = RFR_MODE_CHIRP;
    p->window = *window;
    p->out_flags = RFR_OUT_TONES;
    p->words.assign(start_words, start_words + n_chirps);
    p->rates.assign(rate_words, rate_words + n_chirps);
    cudaGetDevice(&p->device);
    cudaDeviceGetAttribute(&p->n_sms, cudaDevAttrMultiProcessorCount, p->device);
    cudaDeviceGetAttribute(&p->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    p->L = taps;
    p->D = decimation;
    p->h64.resize(taps);
    if (rfr::build_lowpass(window->kind, window->beta, window->cutoff, taps, p->h64.data()) != 0) {
        destroy(p);
        return RFR_E_INVALID;
    }
    p->h32.resize(taps);
    for (int j = 0; j < taps; ++j) p->h32[j] = static_cast<float>(p->h64[j]);
    p->W = taps;
    p->H = decimation;
    p->carry_cap = std::max<int64_t>(taps, 1);
    cudaError_t e = cudaSuccess;
    if ((e = dev_alloc(&p->d_words, static_cast<size_t>(n_chirps) * 8)) != cudaSuccess ||
        (e = dev_alloc(&p->d_rates, static_cast<size_t>(n_chirps) * 8)) != cudaSuccess ||
        (e = dev_alloc(&p->d_h32, static_cast<size_t>(taps) * 4)) != cudaSuccess ||
        (e = dev_alloc(&p->d_status, sizeof(int))) != cudaSuccess ||
        (e = dev_alloc(&p->d_carry[0], static_cast<size_t>(p->carry_cap) * 4)) != cudaSuccess ||
        (e = dev_alloc(&p->d_carry[1], static_cast<size_t>(p->carry_cap) * 4)) != cudaSuccess) {
        const rfr_status st = cuda_fail(p, e, "plan alloc");
        destroy(p);
        return st;
    }
    cudaMemcpy(p->d_words, start_words, static_cast<size_t>(n_chirps) * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_rates, rate_words, static_cast<size_t>(n_chirps) * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_h32, p->h32.data(), static_cast<size_t>(taps) * 4, cudaMemcpyHostToDevice);
    if (reset_state(p) != RFR_OK || cudaDeviceSynchronize() != cudaSuccess) {
        destroy(p);
        return RFR_E_CUDA;
    }
    *out = p;
    return RFR_OK;
}

uint64_t rfr_chirp_rate_word(double k_hz_per_s, double fs_hz) {
    return static_cast<uint64_t>(static_cast<int64_t>(std::llround(std::ldexp(k_hz_per_s / (fs_hz * fs_hz), 64))));
}

rfr_status rfr_chirp_synthesize(uint64_t start_word, uint64_t rate_word, double amplitude, int64_t m0,
                                int64_t n, int16_t* iq_out, void* stream) {
    rfr::TraceRange tr("rfr_chirp_synthesize");
    if (n < 0 || (n > 0 && !iq_out) || !(amplitude >= 0.0) || amplitude > 32767.0) return RFR_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (rfr::chirp_synth(start_word, rate_word, amplitude, m0, n, iq_out, st) != cudaSuccess) return RFR_E_CUDA;
    if (rfr::debug_sync_allowed(st) && (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess))
        return RFR_E_CUDA;
    return RFR_OK;
}

void rfr_plan_destroy(rfr_plan* p) { destroy(p); }

rfr_status rfr_plan_get_info(const rfr_plan* p, rfr_plan_info* info) {
    if (!p || !info) return RFR_E_INVALID;
    info->mode = p->mode;
    info->channels = p->N;
    info->taps = p->mode == RFR_MODE_PFB ? p->T : p->L;   // L for demodulation and chirps
    info->decimation = static_cast<int32_t>(p->H);
    info->n_tones = static_cast<int32_t>(p->words.size());
    info->out_flags = p->out_flags;
    info->samples_consumed = p->samples;
    info->frames_produced = p->frames;
    info->frames_pending = p->q_frames;
    info->tap_scale = p->mode == RFR_MODE_DEMOD ? std::ldexp(1.0, p->tap_exp) : 1.0;
    return RFR_OK;
}

rfr_status rfr_frames_for(const rfr_plan* p, int64_t n, int64_t* frames) {
    if (!p || !frames || n < 0) return RFR_E_INVALID;
    *frames = frames_for_len(p, p->cl + n);
    return RFR_OK;
}

rfr_status rfr_push_into(rfr_plan* p, const int16_t* iq, int64_t n, rfr_output* out, void* stream) {
    rfr::TraceRange tr("rfr_push_into");
    if (!p || !out) return RFR_E_INVALID;
    int64_t F = 0;
    rfr_status s = push_core(p, iq, n, out, &F, static_cast<cudaStream_t>(stream));
    if (s == RFR_OK) s = debug_check(p, static_cast<cudaStream_t>(stream), "rfr_push_into");
    out->frames = (s == RFR_OK) ? F : 0;
    return s;
}

rfr_status rfr_push(rfr_plan* p, const int16_t* iq, int64_t n, void* stream) {
    rfr::TraceRange tr("rfr_push");
    if (!p) return RFR_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t F = frames_for_len(p, p->cl + n);
    const int nt = static_cast<int>(p->words.size());
    const bool want_full = p->mode == RFR_MODE_PFB && (p->out_flags & RFR_OUT_FULL);
    const bool want_tones = nt > 0 && (p->mode == RFR_MODE_DEMOD || (p->out_flags & RFR_OUT_TONES));
    if (p->q_frames + F > p->q_cap) {
        int64_t cap = std::max<int64_t>(p->q_frames + F, 2 * p->q_cap);
        void *nf = nullptr, *nt_ = nullptr;
        if (want_full) RFR_CUDA(p, dev_alloc(&nf, static_cast<size_t>(cap) * p->N * 8));
        if (want_tones) RFR_CUDA(p, dev_alloc(&nt_, static_cast<size_t>(cap) * nt * 8));
        RFR_CUDA(p, cudaStreamSynchronize(st));
        if (p->q_frames > 0) {
            if (want_full)
                RFR_CUDA(p, cudaMemcpy(nf, p->d_qfull, static_cast<size_t>(p->q_frames) * p->N * 8,
                                       cudaMemcpyDeviceToDevice));
            if (want_tones)
                RFR_CUDA(p, cudaMemcpy2D(nt_, cap * 8, p->d_qtones, p->q_cap * 8, p->q_frames * 8, nt,
                                         cudaMemcpyDeviceToDevice));
        }
        dev_free(p->d_qfull);
        dev_free(p->d_qtones);
        p->d_qfull = nf;
        p->d_qtones = nt_;
        p->q_cap = cap;
    }
    rfr_output o{};
    o.full = p->d_qfull;
    o.full_ld = p->N;
    o.full_cap = p->q_cap;
    o.tones = p->d_qtones;
    o.tones_ld = p->q_cap;
    o.tones_cap = p->q_cap;
    o.frame_offset = p->q_frames;
    int64_t got = 0;
    rfr_status s = push_core(p, iq, n, &o, &got, st);
    if (s == RFR_OK) p->q_frames += got;
    if (s == RFR_OK) s = debug_check(p, st, "rfr_push");
    return s;
}

rfr_status rfr_pull(rfr_plan* p, rfr_output* out) {
    rfr::TraceRange tr("rfr_pull");
    if (!p || !out) return RFR_E_INVALID;
    const int64_t F = p->q_frames;
    out->frames = 0;
    if (!out_ok(p, out, F)) return fail(p, RFR_E_SHORT, "pull: output too small");
    cudaStream_t st = p->last_stream;
    const int nt = static_cast<int>(p->words.size());
    if (F > 0) {
        if (p->mode == RFR_MODE_PFB && (p->out_flags & RFR_OUT_FULL))
            RFR_CUDA(p, cudaMemcpy2DAsync(static_cast<char*>(out->full) + out->frame_offset * out->full_ld * 8,
                                          out->full_ld * 8, p->d_qfull, p->N * 8, p->N * 8, F,
                                          cudaMemcpyDefault, st));
        if (nt > 0 && (p->mode == RFR_MODE_DEMOD || (p->out_flags & RFR_OUT_TONES)))
            RFR_CUDA(p, cudaMemcpy2DAsync(static_cast<char*>(out->tones) + out->frame_offset * 8,
                                          out->tones_ld * 8, p->d_qtones, p->q_cap * 8, F * 8, nt,
                                          cudaMemcpyDefault, st));
    }
    RFR_CUDA(p, cudaStreamSynchronize(st));
    rfr_status s = check_status(p);
    if (s != RFR_OK) return s;
    p->q_frames = 0;
    out->frames = F;
    return RFR_OK;
}

rfr_status rfr_process_host(rfr_plan* p, const int16_t* iq_host, int64_t n, rfr_output* out) {
    rfr::TraceRange tr("rfr_process_host");
    if (!p || !out || n < 0 || (n > 0 && !iq_host)) return RFR_E_INVALID;
    const int64_t Ftot = frames_for_len(p, p->cl + n);
    if (!out_ok(p, out, Ftot)) return fail(p, RFR_E_SHORT, "process_host: output too small");
    const int nt = static_cast<int>(p->words.size());
    const bool want_full = p->mode == RFR_MODE_PFB && (p->out_flags & RFR_OUT_FULL);
    const bool want_tones = nt > 0 && (p->mode == RFR_MODE_DEMOD || (p->out_flags & RFR_OUT_TONES));
    // chunk: a multiple of the hop, about 2^24 samples
    const int64_t chunk = std::max<int64_t>(p->H, (int64_t(1) << 24) / p->H * p->H);
    const int64_t fmax = chunk / p->H + 2;
    // A strided device-to-host copy runs at the link's rate only with rows of
    // about 128 KB or more (32 KB rows reach about half of it), so the tone
    // rows of several chunks collect in one group buffer of >= 16384 frames
    // (within 256 MB) and leave in one copy.
    int64_t gcap = fmax;
    if (want_tones) {
        const int64_t by_rows = (16384 + fmax - 1) / fmax;
        const int64_t by_mem = std::max<int64_t>(1, (int64_t(256) << 20) / (static_cast<int64_t>(nt) * 8 * fmax));
        gcap = fmax * std::min(by_rows, by_mem);
    }
    if (p->stage_samples < chunk || (want_tones && p->tgroup_cap < gcap)) {
        cudaDeviceSynchronize();
        for (int i = 0; i < rfr_plan::kStageBufs; ++i) {
            dev_free(p->d_stage_in[i]);
            dev_free(p->d_stage_full[i]);
            p->d_stage_in[i] = p->d_stage_full[i] = nullptr;
        }
        for (auto& g : p->d_tgroup) {
            dev_free(g);
            g = nullptr;
        }
        p->stage_samples = 0;
        p->tgroup_cap = 0;
        for (int i = 0; i < rfr_plan::kStageBufs; ++i) {
            RFR_CUDA(p, dev_alloc(&p->d_stage_in[i], static_cast<size_t>(chunk) * 4));
            if (want_full) RFR_CUDA(p, dev_alloc(&p->d_stage_full[i], static_cast<size_t>(fmax) * p->N * 8));
            if (!p->stage_st[i]) RFR_CUDA(p, cudaStreamCreateWithFlags(&p->stage_st[i], cudaStreamNonBlocking));
        }
        for (auto& e : p->stage_ev)
            if (!e) RFR_CUDA(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        if (want_tones) {
            for (int g = 0; g < rfr_plan::kToneGroups; ++g) {
                RFR_CUDA(p, dev_alloc(&p->d_tgroup[g], static_cast<size_t>(gcap) * nt * 8));
                if (!p->tgroup_ev[g]) RFR_CUDA(p, cudaEventCreateWithFlags(&p->tgroup_ev[g], cudaEventDisableTiming));
            }
            p->tgroup_cap = gcap;
        }
        p->stage_samples = chunk;
    }
    gcap = want_tones ? p->tgroup_cap : gcap;
    int64_t done = 0, fo = out->frame_offset;
    int i = 0;
    cudaEvent_t prev = nullptr;
    int g = 0;                       // tone group being filled
    int64_t gused = 0, gfo = fo;     // its frames so far, its first output frame
    bool g_out[rfr_plan::kToneGroups] = {};   // a copy out of the group buffer is in flight
    while (done < n) {
        const int64_t cnt = std::min(chunk, n - done);
        const int s = i % rfr_plan::kStageBufs;
        cudaStream_t st = p->stage_st[s];
        RFR_CUDA(p, cudaMemcpyAsync(p->d_stage_in[s], iq_host + 2 * done, static_cast<size_t>(cnt) * 4,
                                    cudaMemcpyHostToDevice, st));
        if (prev) RFR_CUDA(p, cudaStreamWaitEvent(st, prev, 0));   // pushes stay in stream order
        if (want_tones && gused == 0 && g_out[g]) RFR_CUDA(p, cudaStreamWaitEvent(st, p->tgroup_ev[g], 0));
        rfr_output o{};
        o.full = p->d_stage_full[s];
        o.full_ld = p->N;
        o.full_cap = fmax;
        if (want_tones) {
            o.tones = static_cast<char*>(p->d_tgroup[g]) + gused * 8;
            o.tones_ld = gcap;
            o.tones_cap = gcap - gused;
        }
        int64_t F = 0;
        rfr_status rs = push_core(p, static_cast<const int16_t*>(p->d_stage_in[s]), cnt, &o, &F, st);
        if (rs != RFR_OK) return rs;
        RFR_CUDA(p, cudaEventRecord(p->stage_ev[s], st));
        prev = p->stage_ev[s];
        if (F > 0 && want_full)
            RFR_CUDA(p, cudaMemcpy2DAsync(static_cast<char*>(out->full) + fo * out->full_ld * 8, out->full_ld * 8,
                                          p->d_stage_full[s], p->N * 8, p->N * 8, F, cudaMemcpyDeviceToHost, st));
        fo += F;
        done += cnt;
        gused += F;
        // the group leaves when the next chunk might not fit, or at the end;
        // every earlier push into it precedes this one in stream order
        if (want_tones && gused > 0 && (gused + fmax > gcap || done == n)) {
            RFR_CUDA(p, cudaMemcpy2DAsync(static_cast<char*>(out->tones) + gfo * 8, out->tones_ld * 8,
                                          p->d_tgroup[g], gcap * 8, gused * 8, nt, cudaMemcpyDeviceToHost, st));
            RFR_CUDA(p, cudaEventRecord(p->tgroup_ev[g], st));
            g_out[g] = true;
            g = (g + 1) % rfr_plan::kToneGroups;
            gused = 0;
            gfo = fo;
        }
        ++i;
    }
    for (int s = 0; s < rfr_plan::kStageBufs; ++s) RFR_CUDA(p, cudaStreamSynchronize(p->stage_st[s]));
    p->last_stream = p->stage_st[(i + rfr_plan::kStageBufs - 1) % rfr_plan::kStageBufs];
    out->frames = fo - out->frame_offset;
    return check_status(p);
}

rfr_status rfr_wait_selftest(int64_t limit_ns, int32_t* device_status) {
    if (limit_ns < 1000 || limit_ns > 2000000000LL) return RFR_E_INVALID;
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return RFR_E_NOMEM;
    cudaMemset(d, 0, sizeof(int));
    wait_selftest_kernel<<<1, 32>>>(d, static_cast<uint64_t>(limit_ns));
    int st = 0;
    const cudaError_t e1 = cudaGetLastError();
    const cudaError_t e2 = cudaMemcpy(&st, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e1 != cudaSuccess || e2 != cudaSuccess) return RFR_E_CUDA;
    if (device_status) *device_status = st;
    return st == DEV_TIMEOUT ? RFR_E_TIMEOUT : RFR_OK;
}

rfr_status rfr_plan_inject_device_status(rfr_plan* p, int32_t status) {
    if (!p || status < DEV_OK || status > rfr::DEV_BADARG) return RFR_E_INVALID;
    RFR_CUDA(p, cudaDeviceSynchronize());
    const int v = status;
    RFR_CUDA(p, cudaMemcpy(p->d_status, &v, sizeof(int), cudaMemcpyHostToDevice));
    return RFR_OK;
}

rfr_status rfr_plan_seek(rfr_plan* p, int64_t start_sample, const int16_t* history, int64_t n_history) {
    if (!p || start_sample < 0 || start_sample % p->H != 0 || n_history < 0) return RFR_E_INVALID;
    const int64_t halo = p->W - p->H;                 // internal window minus hop
    // history the caller provides: N*T - hop (PFB) or L - D (demodulation);
    // the kernel's zero-padded extra taps (if any) see zeros, which they ignore
    const int64_t user_halo = p->mode == RFR_MODE_PFB ? static_cast<int64_t>(p->T) * p->N - p->H
                                                      : static_cast<int64_t>(p->L) - p->D;
    const int64_t want = std::min<int64_t>(std::max<int64_t>(user_halo, 0), start_sample);
    if (n_history != want || (want > 0 && !history))
        return fail(p, RFR_E_INVALID, "seek: history must hold the min(W - hop, start) samples before start");
    RFR_CUDA(p, cudaDeviceSynchronize());
    p->cur = 0;
    p->q_frames = 0;
    p->samples = start_sample;
    p->frames = start_sample / p->H;
    p->cl = halo;                                     // = W - H (may be <= 0 for L <= D)
    if (halo > 0) {
        char* dst = reinterpret_cast<char*>(p->d_carry[0]);
        const int64_t zeros = halo - want;            // before the stream start
        if (zeros > 0) RFR_CUDA(p, cudaMemset(dst, 0, static_cast<size_t>(zeros) * 4));
        if (want > 0)
            RFR_CUDA(p, cudaMemcpy(dst + zeros * 4, history, static_cast<size_t>(want) * 4, cudaMemcpyDefault));
    }
    return RFR_OK;
}

rfr_status rfr_plan_set_demod_products(rfr_plan* p, int32_t products) {
    if (!p || p->mode != RFR_MODE_DEMOD || (products != 3 && products != 4)) return RFR_E_INVALID;
    if (products == 4) {
        p->demod_products = 4;
        p->accum_chunk = 2;
        return RFR_OK;
    }
    if (p->D % 64 != 0) return fail(p, RFR_E_UNSUPPORTED, "the three-product form needs D % 64 == 0");
    if (p->words.empty()) return fail(p, RFR_E_INVALID, "no tones");
    if (!p->d_b3) {
        const int nt = static_cast<int>(p->words.size());
        p->Lpad3 = (p->L + 63) / 64 * 64;
        p->ntp3 = (nt + 127) / 128 * 128;
        p->tap_exp3 = p->tap_exp - 1;      // |ci -+ cr| <= sqrt(2) max|h|
        const size_t plane = static_cast<size_t>(p->ntp3) * p->Lpad3;
        double* d_h64 = nullptr;
        cudaError_t e = dev_alloc(&p->d_b3, plane * 6 * sizeof(uint16_t));
        if (e == cudaSuccess) e = dev_alloc(&d_h64, static_cast<size_t>(p->L) * 8);
        if (e == cudaSuccess) e = cudaMemcpy(d_h64, p->h64.data(), static_cast<size_t>(p->L) * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = rfr::demod3_build_taps(d_h64, p->d_words, nt, p->ntp3, p->L, p->Lpad3, p->tap_exp3, p->d_b3, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        dev_free(d_h64);
        if (e != cudaSuccess) {
            dev_free(p->d_b3);
            p->d_b3 = nullptr;
            return cuda_fail(p, e, "three-product tap build");
        }
    }
    p->demod_products = 3;
    p->accum_chunk = 4;                // 256 taps per TMEM chunk
    return RFR_OK;
}

rfr_status rfr_plan_set_accum_chunk(rfr_plan* p, int32_t k_blocks) {
    if (!p || p->mode != RFR_MODE_DEMOD || k_blocks < 1 || k_blocks > 64) return RFR_E_INVALID;
    p->accum_chunk = k_blocks;
    return RFR_OK;
}

rfr_status rfr_reset(rfr_plan* p) {
    if (!p) return RFR_E_INVALID;
    RFR_CUDA(p, cudaDeviceSynchronize());
    return reset_state(p);
}

// State blob: magic, version, mode, N/L, T/D, W, H, samples, frames, cl,
// then max(cl, 0) carry samples.
namespace {
struct StateHeader {
    uint32_t magic, version;
    int32_t mode, a, b, pad;
    int64_t W, H, samples, frames, cl;
};
constexpr uint32_t kStateMagic = 0x52465253;  // "RFRS"
}  // namespace

rfr_status rfr_state_export(rfr_plan* p, void* host, size_t* bytes) {
    if (!p || !bytes) return RFR_E_INVALID;
    const int64_t keep = std::max<int64_t>(p->cl, 0);
    const size_t need = sizeof(StateHeader) + static_cast<size_t>(keep) * 4;
    if (!host) {
        *bytes = need;
        return RFR_OK;
    }
    if (*bytes < need) {
        *bytes = need;
        return fail(p, RFR_E_SHORT, "state buffer too small");
    }
    RFR_CUDA(p, cudaDeviceSynchronize());
    StateHeader h{kStateMagic, 1, p->mode, p->mode == RFR_MODE_PFB ? p->N : p->L,
                  p->mode == RFR_MODE_PFB ? p->T : p->D, 0, p->W, p->H, p->samples, p->frames, p->cl};
    std::memcpy(host, &h, sizeof(h));
    if (keep > 0)
        RFR_CUDA(p, cudaMemcpy(static_cast<char*>(host) + sizeof(h), p->d_carry[p->cur],
                               static_cast<size_t>(keep) * 4, cudaMemcpyDeviceToHost));
    *bytes = need;
    return RFR_OK;
}

rfr_status rfr_state_import(rfr_plan* p, const void* host, size_t bytes) {
    if (!p || !host || bytes < sizeof(StateHeader)) return RFR_E_INVALID;
    StateHeader h;
    std::memcpy(&h, host, sizeof(h));
    if (h.magic != kStateMagic || h.version != 1 || h.mode != p->mode ||
        h.a != (p->mode == RFR_MODE_PFB ? p->N : p->L) || h.b != (p->mode == RFR_MODE_PFB ? p->T : p->D) ||
        h.W != p->W || h.H != p->H)
        return fail(p, RFR_E_INVALID, "state does not match this plan");
    const int64_t keep = std::max<int64_t>(h.cl, 0);
    if (keep > p->carry_cap || bytes < sizeof(h) + static_cast<size_t>(keep) * 4)
        return fail(p, RFR_E_INVALID, "state blob truncated");
    RFR_CUDA(p, cudaDeviceSynchronize());
    p->cur = 0;
    if (keep > 0)
        RFR_CUDA(p, cudaMemcpy(p->d_carry[0], static_cast<const char*>(host) + sizeof(h),
                               static_cast<size_t>(keep) * 4, cudaMemcpyHostToDevice));
    p->samples = h.samples;
    p->frames = h.frames;
    p->cl = h.cl;
    p->q_frames = 0;
    return RFR_OK;
}

rfr_status rfr_plan_get_taps(const rfr_plan* p, double* h64, float* h32, int64_t* n) {
    if (!p || !n) return RFR_E_INVALID;
    *n = static_cast<int64_t>(p->h64.size());
    if (h64) std::memcpy(h64, p->h64.data(), p->h64.size() * 8);
    if (h32) std::memcpy(h32, p->h32.data(), p->h32.size() * 4);
    return RFR_OK;
}

rfr_status rfr_plan_get_bins(const rfr_plan* p, int32_t* bins, int32_t* count) {
    if (!p || !count) return RFR_E_INVALID;
    *count = static_cast<int32_t>(p->bins.size());
    if (bins && !p->bins.empty()) std::memcpy(bins, p->bins.data(), p->bins.size() * 4);
    return RFR_OK;
}

rfr_status rfr_plain_oneshot(rfr_plan* p, const int16_t* iq, int64_t n, rfr_output* out, void* stream) {
    return rfr_plain_oneshot_form(p, RFR_PLAIN_DEFAULT, iq, n, out, stream);
}

rfr_status rfr_plain_oneshot_form(rfr_plan* p, int32_t form, const int16_t* iq, int64_t n, rfr_output* out,
                                  void* stream) {
    rfr::TraceRange tr("rfr_plain_oneshot");
    if (!p || !out || n < 0 || (n > 0 && !iq)) return RFR_E_INVALID;
    if (form != RFR_PLAIN_DEFAULT && form != RFR_PLAIN_CGEMM) return fail(p, RFR_E_INVALID, "unknown plain form");
    if (p->mode == RFR_MODE_CHIRP) return fail(p, RFR_E_UNSUPPORTED, "no plain form for chirp plans");
    if (form == RFR_PLAIN_CGEMM && p->mode != RFR_MODE_DEMOD)
        return fail(p, RFR_E_UNSUPPORTED, "the Cgemm form is a demodulation form");
    if (p->mode == RFR_MODE_PFB && p->H != p->N)
        return fail(p, RFR_E_UNSUPPORTED, "the plain form is critically sampled only");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // zero history: frame k uses samples ((k+1)*hop - W, (k+1)*hop]
    const int64_t W = p->mode == RFR_MODE_PFB ? static_cast<int64_t>(p->N) * p->T : p->L;
    const int64_t F = n / p->H;
    (void)W;
    if (!out_ok(p, out, F)) return fail(p, RFR_E_SHORT, "plain: output too small");
    const int nt = static_cast<int>(p->words.size());
    if (F > 0) {
        if (p->mode == RFR_MODE_PFB) {
            const bool tones = (p->out_flags & RFR_OUT_TONES) != 0;
            RFR_CUDA(p, rfr::plain_pfb(iq, n, p->N, p->T, p->d_h32, p->d_bins, tones ? nt : 0,
                                       (p->out_flags & RFR_OUT_FULL) ? static_cast<char*>(out->full) + out->frame_offset * out->full_ld * 8 : nullptr,
                                       out->full_ld,
                                       tones ? static_cast<char*>(out->tones) + out->frame_offset * 8 : nullptr,
                                       out->tones_ld, &p->plain_scratch, &p->plain_scratch_bytes,
                                       &p->plain_fft, &p->plain_fft_batch, st));
        } else if (nt > 0) {
            if (!p->d_c32) {
                RFR_CUDA(p, dev_alloc(&p->d_c32, static_cast<size_t>(nt) * p->L * 8));
                RFR_CUDA(p, rfr::plain_demod_taps(p->d_h32, p->d_words, nt, p->L, p->d_c32, st));
            }
            char* t0 = static_cast<char*>(out->tones) + out->frame_offset * 8;
            if (form == RFR_PLAIN_CGEMM)
                RFR_CUDA(p, rfr::plain_demod_cgemm(iq, n, p->L, p->D, p->d_c32, p->d_words, nt, t0, out->tones_ld,
                                                   &p->plain_scratch, &p->plain_scratch_bytes, &p->plain_blas, st));
            else
                RFR_CUDA(p, rfr::plain_demod(iq, n, p->L, p->D, p->d_c32, p->d_words, nt, t0, out->tones_ld, st));
        }
    }
    out->frames = F;
    return RFR_OK;
}

}  // extern "C"
