// batch.cu -- many readout streams per step (the batched workload), and the
// launch autotuner.
//
// rfr_batch_push enqueues one push per plan.  Each plan's kernels go on its
// own branch (fork/join with events), except the demodulation GEMMs of the
// three-product plans: those of all plans run as ONE persistent kernel launch
// over every plan's tiles (demod3_gemm), after the plans' pre-GEMM kernels.
// The whole step is captured into a CUDA graph and launched into the caller's
// stream as ONE graph launch.
// The executable graph is kept and updated in place (cudaGraphExecUpdate) on
// the next step, so steady-state steps re-instantiate nothing.  Allocation
// (scratch growth) happens before capture, never inside it.
//
// rfr_plan_autotune times the launch choices that never change results
// (bit-identical outputs) -- the PFB ring look-ahead, and the demodulation
// GEMM's tile raster and tone-tile width (128 or 64 tones per tile) -- on a
// buffer of the caller's size, keeps the fastest in the plan and in a
// JSON cache file (RFR_TUNE_CACHE, default ./rfr_tune_cache.json) keyed by
// the plan shape and the GPU, so later plans of the same shape load it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "rfr_internal.h"
#include "trace.h"

struct rfr_batch {
    std::vector<rfr_plan*> plans;
    std::vector<cudaStream_t> branches;
    std::vector<cudaEvent_t> ev_join;
    std::vector<rfr::DemodGemmJob> jobs;   // deferred three-product GEMMs, one per plan
    cudaStream_t origin = nullptr;
    cudaStream_t gemm_stream = nullptr;    // the persistent GEMM launch of the step
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_gemm = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t steps = 0, updates = 0, instantiations = 0;
    std::string last_error;
};

namespace {

rfr_status batch_fail(rfr_batch* b, rfr_status s, const std::string& msg) {
    if (b) b->last_error = msg;
    return s;
}

void batch_destroy(rfr_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto s : b->branches) cudaStreamDestroy(s);
    for (auto e : b->ev_join) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_gemm) cudaEventDestroy(b->ev_gemm);
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->gemm_stream) cudaStreamDestroy(b->gemm_stream);
    delete b;
}

// ------------------------------------------------------------ tune cache
std::mutex g_tune_mu;

std::string tune_path() {
    const char* p = std::getenv("RFR_TUNE_CACHE");
    return p && *p ? std::string(p) : std::string("rfr_tune_cache.json");
}

std::string tune_key(const rfr_plan* p, int64_t n) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, p->device);
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= n) ++lg;
    std::ostringstream k;
    k << (p->mode == RFR_MODE_PFB ? "pfb" : "demod") << ":N" << p->N << ":T" << p->T << ":L" << p->L
      << ":D" << p->D << ":tones" << p->words.size() << ":flags" << p->out_flags << ":n2^" << lg
      << ":sm" << prop.major << prop.minor << "x" << prop.multiProcessorCount;
    return k.str();
}

// Minimal line-oriented JSON map:
//   {"key": [pfb_lookahead, demod_raster, demod_tone_tile, demod_fused], ...}
// (missing trailing numbers take their defaults: tone tile 128, not fused)
struct TuneEntry {
    int lookahead = 0, raster = 1, bt = 128, fused = 0, pair = 0, cluster = 0;
};
std::map<std::string, TuneEntry> tune_load() {
    std::map<std::string, TuneEntry> m;
    std::ifstream f(tune_path());
    std::string line;
    while (std::getline(f, line)) {
        const size_t q0 = line.find('"'), q1 = line.find('"', q0 + 1);
        const size_t b0 = line.find('[', q1 == std::string::npos ? 0 : q1);
        if (q0 == std::string::npos || q1 == std::string::npos || b0 == std::string::npos) continue;
        TuneEntry t;
        const int got = std::sscanf(line.c_str() + b0, "[%d, %d, %d, %d, %d, %d]", &t.lookahead, &t.raster, &t.bt,
                                    &t.fused, &t.pair, &t.cluster);
        if (got >= 2) {
            if (got == 2 || (t.bt != 64 && t.bt != 128)) t.bt = 128;
            if (got < 4 || (t.fused != 0 && t.fused != 1)) t.fused = 0;
            if (got < 5 || (t.pair != 0 && t.pair != 1) || t.fused) t.pair = 0;
            if (got < 6 || (t.cluster != 0 && t.cluster != 1)) t.cluster = 0;
            m[line.substr(q0 + 1, q1 - q0 - 1)] = t;
        }
    }
    return m;
}

void tune_store(const std::map<std::string, TuneEntry>& m) {
    const std::string path = tune_path(), tmp = path + ".tmp";
    {
        std::ofstream f(tmp);
        f << "{\n";
        size_t i = 0;
        for (const auto& kv : m) {
            f << "  \"" << kv.first << "\": [" << kv.second.lookahead << ", " << kv.second.raster << ", "
              << kv.second.bt << ", " << kv.second.fused << ", " << kv.second.pair << ", " << kv.second.cluster << "]"
              << (++i < m.size() ? "," : "") << "\n";
        }
        f << "}\n";
    }
    std::rename(tmp.c_str(), path.c_str());
}

}  // namespace

extern "C" {

rfr_status rfr_batch_create(rfr_batch** out, rfr_plan* const* plans, int32_t n) {
    if (!out || !plans || n < 1 || n > 4096) return RFR_E_INVALID;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return RFR_E_INVALID;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return RFR_E_INVALID;   // a plan's pushes must stay ordered
    }
    rfr_batch* b = new (std::nothrow) rfr_batch();
    if (!b) return RFR_E_NOMEM;
    b->plans.assign(plans, plans + n);
    const int nb = std::min(n, 32);
    b->branches.resize(nb, nullptr);
    b->ev_join.resize(n, nullptr);
    b->jobs.resize(n);
    bool ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->gemm_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_gemm, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (auto& s : b->branches) ok = ok && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    for (auto& e : b->ev_join) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        batch_destroy(b);
        return RFR_E_CUDA;
    }
    *out = b;
    return RFR_OK;
}

void rfr_batch_destroy(rfr_batch* b) {
    if (b) cudaDeviceSynchronize();
    batch_destroy(b);
}

rfr_status rfr_batch_push(rfr_batch* b, const int16_t* const* bufs, const int64_t* n_samples,
                          rfr_output* outs, void* stream) {
    rfr::TraceRange tr("rfr_batch_push");
    if (!b || !bufs || !n_samples || !outs) return RFR_E_INVALID;
    const int n = static_cast<int>(b->plans.size());
    // 1. validate and grow scratch outside of any capture
    for (int i = 0; i < n; ++i) {
        rfr_plan* p = b->plans[i];
        rfr_status s = rfr::push_check(p, bufs[i], n_samples[i], &outs[i]);
        if (s != RFR_OK) return batch_fail(b, s, "push " + std::to_string(i) + ": " + p->last_error);
        s = rfr::ensure_scratch(p, n_samples[i]);
        if (s != RFR_OK) return batch_fail(b, s, "scratch: " + p->last_error);
    }
    // 2. capture the step: fork one branch per plan, join back
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return batch_fail(b, RFR_E_CUDA, "begin capture");
    rfr_status err = RFR_OK;
    cudaEventRecord(b->ev_fork, b->origin);
    cudaStreamWaitEvent(b->gemm_stream, b->ev_fork, 0);
    std::vector<const rfr::DemodGemmJob*> gemms;
    for (int i = 0; i < n && err == RFR_OK; ++i) {
        cudaStream_t br = b->branches[i % b->branches.size()];
        cudaStreamWaitEvent(br, b->ev_fork, 0);
        int64_t F = 0;
        err = rfr::push_core(b->plans[i], bufs[i], n_samples[i], &outs[i], &F, br, &b->jobs[i]);
        outs[i].frames = F;
        if (err != RFR_OK) b->last_error = "push " + std::to_string(i) + ": " + b->plans[i]->last_error;
        cudaEventRecord(b->ev_join[i], br);
        if (b->jobs[i].n_tiles > 0) {
            // the plan's GEMM waits for its pre-GEMM kernels
            cudaStreamWaitEvent(b->gemm_stream, b->ev_join[i], 0);
            gemms.push_back(&b->jobs[i]);
        } else {
            cudaStreamWaitEvent(b->origin, b->ev_join[i], 0);
        }
    }
    if (err == RFR_OK && !gemms.empty()) {
        const cudaError_t ge = rfr::demod3_gemm(gemms.data(), static_cast<int>(gemms.size()), b->plans[0]->n_sms,
                                                b->gemm_stream);
        if (ge != cudaSuccess) {
            err = RFR_E_CUDA;
            b->last_error = std::string("batched GEMM launch: ") + cudaGetErrorString(ge);
        }
    }
    cudaEventRecord(b->ev_gemm, b->gemm_stream);
    cudaStreamWaitEvent(b->origin, b->ev_gemm, 0);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->origin, &graph);
    if (err != RFR_OK) {
        // only a CUDA error can get here (arguments were checked above); the
        // plans' stream state is no longer meaningful: reset them before reuse
        if (graph) cudaGraphDestroy(graph);
        return err;
    }
    if (ce != cudaSuccess || !graph) return batch_fail(b, RFR_E_CUDA, "end capture");
    // 3. update the executable graph in place, or instantiate it
    bool updated = false;
    if (b->exec) {
        cudaGraphExecUpdateResultInfo info{};
        if (cudaGraphExecUpdate(b->exec, graph, &info) == cudaSuccess) {
            updated = true;
            ++b->updates;
        } else {
            cudaGetLastError();
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
    }
    if (!updated) {
        if (cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
            cudaGraphDestroy(graph);
            return batch_fail(b, RFR_E_CUDA, "graph instantiate");
        }
        ++b->instantiations;
    }
    cudaGraphDestroy(graph);
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return batch_fail(b, RFR_E_CUDA, "graph launch");
    for (auto* p : b->plans) p->last_stream = st;
    ++b->steps;
    if (rfr::debug_sync_allowed(st) && (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess))
        return batch_fail(b, RFR_E_CUDA, "RFR_DEBUG: batch step failed on the device");
    return RFR_OK;
}

rfr_status rfr_batch_stats(const rfr_batch* b, int64_t* steps, int64_t* graph_updates,
                           int64_t* graph_instantiations) {
    if (!b) return RFR_E_INVALID;
    if (steps) *steps = b->steps;
    if (graph_updates) *graph_updates = b->updates;
    if (graph_instantiations) *graph_instantiations = b->instantiations;
    return RFR_OK;
}

const char* rfr_batch_last_error(const rfr_batch* b) { return b ? b->last_error.c_str() : ""; }

rfr_status rfr_plan_autotune(rfr_plan* p, int64_t n_samples, int32_t use_cache, double* best_ms) {
    rfr::TraceRange tr("rfr_plan_autotune");
    if (!p || n_samples < 1 || n_samples > (int64_t(1) << 31)) return RFR_E_INVALID;
    const std::string key = tune_key(p, n_samples);
    if (use_cache) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto m = tune_load();
        auto it = m.find(key);
        if (it != m.end()) {
            p->tune.pfb_lookahead = it->second.lookahead;
            p->tune.demod_raster = it->second.raster;
            p->tune.demod_bt = it->second.bt;
            p->tune.demod_fused = it->second.fused;
            p->tune.demod_pair = it->second.pair;
            p->tune.pfb_cluster = p->d_tw_cl ? it->second.cluster : 0;
            p->tune.tuned = true;
            if (best_ms) *best_ms = -1.0;
            return RFR_OK;
        }
    }
    // candidates (all give bit-identical results)
    std::vector<TuneEntry> cand;
    if (p->mode == RFR_MODE_PFB) {
        for (int la : {1, 2, 3}) cand.push_back({la, 1, 128});
        // N = 8192, 16384 with T <= 8: the cluster kernel beside the direct one
        if (p->d_tw_cl) cand.push_back({0, 1, 128, 0, 0, 1});
    } else {
        // the fused pre-split converts each A tile once per tone tile and
        // product (3 x tone tiles times per sample): timed only for plans of
        // at most two 128-tone tiles, where that stays cheap
        const bool try_fused = p->demod_products == 3 && p->words.size() <= 256;
        for (int fused : {0, 1})
            for (int pair : {1, 0})
                for (int bt : {128, 64}) {
                    // tone tile, fused pre-split and clusters are three-product choices;
                    // the cluster form loads A by TMA, so it excludes the fused pre-split
                    if ((bt == 64 || fused || pair) && p->demod_products != 3) continue;
                    if (fused && (!try_fused || pair)) continue;
                    for (int r : {1, 8, 19, 38}) cand.push_back({0, r, bt, fused, pair});
                }
    }
    // scratch buffers: zero input, outputs sized for the push
    const int64_t F = rfr::frames_for_samples(p, n_samples) + 1;
    const int nt = static_cast<int>(p->words.size());
    void *x = nullptr, *full = nullptr, *tones = nullptr;
    const bool want_full = p->mode == RFR_MODE_PFB && (p->out_flags & RFR_OUT_FULL);
    const bool want_tones = nt > 0 && (p->mode == RFR_MODE_DEMOD || (p->out_flags & RFR_OUT_TONES));
    auto cleanup = [&]() {
        if (x) cudaFree(x);
        if (full) cudaFree(full);
        if (tones) cudaFree(tones);
    };
    if (cudaMalloc(&x, static_cast<size_t>(n_samples) * 4) != cudaSuccess ||
        (want_full && cudaMalloc(&full, static_cast<size_t>(F) * p->N * 8) != cudaSuccess) ||
        (want_tones && cudaMalloc(&tones, static_cast<size_t>(F) * nt * 8) != cudaSuccess)) {
        cleanup();
        return RFR_E_NOMEM;
    }
    cudaMemset(x, 0, static_cast<size_t>(n_samples) * 4);
    // time on a scratch copy of the stream state, then restore it
    const int64_t s_samples = p->samples, s_frames = p->frames, s_cl = p->cl;
    const int s_cur = p->cur;
    std::vector<unsigned char> carry_save(static_cast<size_t>(std::max<int64_t>(p->cl, 0)) * 4);
    if (!carry_save.empty())
        cudaMemcpy(carry_save.data(), p->d_carry[p->cur], carry_save.size(), cudaMemcpyDeviceToHost);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    rfr_output o{};
    o.full = full;
    o.full_ld = p->N;
    o.full_cap = F;
    o.tones = tones;
    o.tones_ld = F;
    o.tones_cap = F;
    const rfr::TuneConfig keep = p->tune;
    double best = 1e30;
    TuneEntry best_c = cand.front();
    rfr_status rs = rfr::ensure_scratch(p, n_samples);
    for (size_t c = 0; c < cand.size() && rs == RFR_OK; ++c) {
        p->tune.pfb_lookahead = cand[c].lookahead;
        p->tune.demod_raster = cand[c].raster;
        p->tune.demod_bt = cand[c].bt;
        p->tune.demod_fused = cand[c].fused;
        p->tune.demod_pair = cand[c].pair;
        p->tune.pfb_cluster = cand[c].cluster;
        float ms_best = 1e30f;
        for (int rep = 0; rep < 4 && rs == RFR_OK; ++rep) {
            p->samples = s_samples;
            p->frames = s_frames;
            p->cl = s_cl;
            p->cur = s_cur;
            cudaEventRecord(e0, st);
            int64_t got = 0;
            rs = rfr::push_core(p, static_cast<const int16_t*>(x), n_samples, &o, &got, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_best = std::min(ms_best, ms);   // first run warms up
        }
        if (ms_best < best) {
            best = ms_best;
            best_c = cand[c];
        }
    }
    // restore the stream state (the carry may have been rewritten)
    p->samples = s_samples;
    p->frames = s_frames;
    p->cl = s_cl;
    p->cur = s_cur;
    if (!carry_save.empty())
        cudaMemcpy(p->d_carry[p->cur], carry_save.data(), carry_save.size(), cudaMemcpyHostToDevice);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cleanup();
    if (rs != RFR_OK) {
        p->tune = keep;
        return rs;
    }
    p->tune.pfb_lookahead = best_c.lookahead;
    p->tune.demod_raster = best_c.raster;
    p->tune.demod_bt = best_c.bt;
    p->tune.demod_fused = best_c.fused;
    p->tune.demod_pair = best_c.pair;
    p->tune.pfb_cluster = best_c.cluster;
    p->tune.tuned = true;
    if (best_ms) *best_ms = best;
    if (use_cache) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto m = tune_load();
        m[key] = best_c;
        tune_store(m);
    }
    return RFR_OK;
}

rfr_status rfr_plan_set_tone_tile(rfr_plan* p, int32_t tones_per_tile) {
    if (!p || p->mode != RFR_MODE_DEMOD || p->demod_products != 3 || (tones_per_tile != 64 && tones_per_tile != 128))
        return RFR_E_INVALID;
    p->tune.demod_bt = tones_per_tile;
    return RFR_OK;
}

rfr_status rfr_plan_set_fused_presplit(rfr_plan* p, int32_t on) {
    if (!p || p->mode != RFR_MODE_DEMOD || p->demod_products != 3 || (on != 0 && on != 1)) return RFR_E_INVALID;
    p->tune.demod_fused = on;
    return RFR_OK;
}

rfr_status rfr_plan_get_fused_presplit(const rfr_plan* p, int32_t* on) {
    if (!p || !on) return RFR_E_INVALID;
    *on = p->mode == RFR_MODE_DEMOD && p->demod_products == 3 ? p->tune.demod_fused : 0;
    return RFR_OK;
}

rfr_status rfr_plan_set_demod_pair(rfr_plan* p, int32_t on) {
    if (!p || p->mode != RFR_MODE_DEMOD || p->demod_products != 3 || (on != 0 && on != 1)) return RFR_E_INVALID;
    p->tune.demod_pair = on;
    return RFR_OK;
}

rfr_status rfr_plan_get_demod_pair(const rfr_plan* p, int32_t* on) {
    if (!p || !on) return RFR_E_INVALID;
    *on = p->mode == RFR_MODE_DEMOD && p->demod_products == 3 && !p->tune.demod_fused ? p->tune.demod_pair : 0;
    return RFR_OK;
}

rfr_status rfr_plan_set_pfb_cluster(rfr_plan* p, int32_t on) {
    if (!p || p->mode != RFR_MODE_PFB || !p->d_tw_cl || (on != 0 && on != 1)) return RFR_E_INVALID;
    p->tune.pfb_cluster = on;
    return RFR_OK;
}

rfr_status rfr_plan_get_pfb_cluster(const rfr_plan* p, int32_t* on) {
    if (!p || !on) return RFR_E_INVALID;
    *on = p->mode == RFR_MODE_PFB && p->d_tw_cl ? p->tune.pfb_cluster : 0;
    return RFR_OK;
}

rfr_status rfr_plan_get_tone_tile(const rfr_plan* p, int32_t* tones_per_tile) {
    if (!p || !tones_per_tile) return RFR_E_INVALID;
    *tones_per_tile = p->mode == RFR_MODE_DEMOD && p->demod_products == 3 ? p->tune.demod_bt : 0;
    return RFR_OK;
}

rfr_status rfr_plan_get_tune(const rfr_plan* p, int32_t* pfb_lookahead, int32_t* demod_raster, int32_t* tuned) {
    if (!p) return RFR_E_INVALID;
    if (pfb_lookahead) *pfb_lookahead = p->tune.pfb_lookahead;
    if (demod_raster) *demod_raster = p->tune.demod_raster;
    if (tuned) *tuned = p->tune.tuned ? 1 : 0;
    return RFR_OK;
}

}  // extern "C"
