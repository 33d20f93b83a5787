// Batches: many independent annealing instances (each its own context, tables
// and trajectories, sizes N = 2 .. 512 mixed) propagated by one persistent
// launch per kernel form, replayed as one CUDA graph.
//
// The trajectories of every instance are independent (arXiv:1710.03431,
// Sec. VI.C: the trajectory method parallelises over trajectories with no
// communication), so a batch is a list of work items (instance, tile of TT
// trajectories) that persistent CTAs take from a queue, longest first. The
// kernel forms: SIMT FP64, SIMT FP32 (every N) and tensor cores (split FP16,
// N = 128 or 256; one launch per N). Tile shapes come from a small
// autotuner: for each form it times the candidate shapes on the batch itself
// over the first grid steps and keeps the fastest; the choice is cached per
// (device, form, instance sizes) for the life of the process.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "aqt_internal.h"

namespace aqt {
// exported by capi.cpp / propagate_tc.cu
int tc_shape(int N, int64_t M, int num_sms);
}  // namespace aqt

namespace {

using namespace aqt;

// kernel forms, one persistent launch each
enum Form : int { kFormF64 = 0, kFormF32 = 1, kFormTc128 = 2, kFormTc256 = 3, kForms = 4 };

constexpr int kSimtThreads = 256;
constexpr int kMaxSimtCtaPerSm = 4;  // scratch is sized for at most this many resident SIMT CTAs per SM
constexpr int kTuneSteps = 33;       // grid points of a tuning run

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int form_of(const BatchMember &m) {
    if (m.precision == AQT_PREC_FP64) return kFormF64;
    if (m.precision == AQT_PREC_FP32) return kFormF32;
    return m.p.N == 128 ? kFormTc128 : kFormTc256;
}

bool is_tc(int f) { return f >= kFormTc128; }

// Trajectories per tile of an instance for a SIMT candidate RA: the largest
// power of two in [4, 64] whose rotation rows per thread fit RA and whose
// states fit shared memory; -1 if none.
int simt_tt(int N, int precision, int RA) {
    for (int tt = 64; tt >= 4; tt >>= 1)
        if (simt_rows_per_thread(N, tt) <= RA && simt_smem_bytes(N, tt, precision) <= kSimtSmemLimit) return tt;
    return -1;
}

// Trajectories per tile of an instance for a tensor-core candidate cap: M
// split evenly into tiles of at most `cap` (a multiple of 8).
int tc_tt(int64_t M, int cap) {
    const int64_t tiles = (M + cap - 1) / cap;
    int tt = (int)((M + tiles - 1) / tiles);
    tt = (tt + 7) & ~7;
    return std::max(8, std::min(tt, cap));
}

std::mutex g_cache_mu;
std::map<std::string, int> g_tune_cache;  // signature -> chosen candidate

}  // namespace

struct aqt_batch {
    int device = -1, num_sms = 0;
    std::string err;
    std::vector<aqt_ctx *> ctx;
    std::vector<BatchMember> mem;
    std::vector<int> form;
    // per form: member indices, candidates, the chosen candidate
    std::vector<int> members[kForms];
    std::vector<int> cands[kForms];
    int chosen[kForms] = {-1, -1, -1, -1};
    bool tuned = false;
    // per member: shape of the chosen candidate
    std::vector<int> TT, n_tiles;
    // workspace layout (caller-owned device memory)
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0, need = 0;
    size_t off_params = 0, off_items = 0, off_queue = 0;
    std::vector<size_t> off_obs;  // per member
    size_t off_scr[kForms] = {0, 0, 0, 0}, scr_stride[kForms] = {0, 0, 0, 0};
    int max_cta[kForms] = {0, 0, 0, 0};
    size_t n_items_max = 0;
    // the graph of one run
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int max_K = 0;
};

namespace {

aqt_status bfail(aqt_batch *b, aqt_status s, const std::string &m) {
    if (b) b->err = m;
    return s;
}

aqt_status bcuda(aqt_batch *b, cudaError_t e, const char *what) {
    return bfail(b, AQT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Shapes of every member of form f under candidate c (TT, tiles); false if
// the candidate does not fit some member.
bool shapes_for(const aqt_batch *b, int f, int c, std::vector<int> &TT, std::vector<int> &tiles) {
    for (int i : b->members[f]) {
        const BatchMember &m = b->mem[i];
        int tt = is_tc(f) ? tc_tt(m.p.M, c) : simt_tt(m.p.N, m.precision, c);
        if (tt <= 0) return false;
        TT[i] = tt;
        tiles[i] = (int)((m.p.M + tt - 1) / tt);
    }
    return true;
}

// Dynamic shared memory of form f's persistent CTA for the given shapes, and
// (tensor cores) the offset of its per-CTA words.
size_t form_smem(const aqt_batch *b, int f, const std::vector<int> &TT, uint32_t *tail) {
    size_t smem = 0;
    *tail = 0;
    if (is_tc(f)) {
        int tt_max = 8;
        for (int i : b->members[f]) tt_max = std::max(tt_max, TT[i]);
        return tc_batch_smem_bytes(f == kFormTc128 ? 128 : 256, tt_max, tail);
    }
    for (int i : b->members[f])
        smem = std::max(smem, simt_smem_bytes(b->mem[i].p.N, TT[i], b->mem[i].precision));
    return smem;
}

int form_occupancy(int f, int RA, size_t smem) {
    if (is_tc(f)) return 1;
    const int nb = f == kFormF64 ? simt_batch_occupancy_f64(RA, smem) : simt_batch_occupancy_f32(RA, smem);
    return std::min(nb, kMaxSimtCtaPerSm);
}

// Work items of form f, longest first: cost ~ N^2 (rotation) x TT x steps.
std::vector<BatchItem> form_items(const aqt_batch *b, int f, const std::vector<int> &TT,
                                  const std::vector<int> &tiles) {
    struct Ord {
        double cost;
        BatchItem it;
    };
    std::vector<Ord> v;
    for (int i : b->members[f]) {
        const BatchMember &m = b->mem[i];
        const double cost = (double)m.p.N * m.p.N * TT[i] * (m.p.K - 1) + 1.0;
        for (int t = 0; t < tiles[i]; ++t) v.push_back({cost, BatchItem{i, t}});
    }
    std::stable_sort(v.begin(), v.end(), [](const Ord &x, const Ord &y) { return x.cost > y.cost; });
    std::vector<BatchItem> out;
    for (auto &o : v) out.push_back(o.it);
    return out;
}

std::string signature(const aqt_batch *b, int f) {
    std::string s = std::to_string(b->device) + "/" + std::to_string(f);
    std::vector<std::string> parts;
    for (int i : b->members[f]) {
        const RunParams &p = b->mem[i].p;
        parts.push_back(std::to_string(p.N) + "x" + std::to_string(p.M) + "x" + std::to_string(p.K));
    }
    std::sort(parts.begin(), parts.end());
    for (auto &x : parts) s += "/" + x;
    return s;
}

// Run parameters of every member for the given shapes (K_run grid points; 0 =
// the member's own), pointing the observable partials and scratch at the
// batch's workspace.
std::vector<RunParams> member_params(const aqt_batch *b, const std::vector<int> &TT, const std::vector<int> &tiles,
                                     int K_run) {
    std::vector<RunParams> ps(b->mem.size());
    for (size_t i = 0; i < b->mem.size(); ++i) {
        RunParams p = b->mem[i].p;
        p.TT = TT[i];
        p.n_cta = tiles[i];
        p.RA = is_tc(b->form[i]) ? 0 : simt_rows_per_thread(p.N, TT[i]);
        if (K_run > 0) p.K = std::min(p.K, K_run);
        p.obs_part = reinterpret_cast<double *>(b->ws + b->off_obs[i]);
        p.scratch = reinterpret_cast<double *>(b->ws + b->off_scr[b->form[i]]);
        ps[i] = p;
    }
    return ps;
}

// Launch description of form f (after the params and items are on the device).
BatchLaunch form_launch(const aqt_batch *b, int f, int cand, const std::vector<int> &TT, size_t item_off,
                        int n_items) {
    BatchLaunch L;
    L.params = reinterpret_cast<const RunParams *>(b->ws + b->off_params);
    L.items = reinterpret_cast<const BatchItem *>(b->ws + b->off_items) + item_off;
    L.n_items = n_items;
    L.queue = reinterpret_cast<int *>(b->ws + b->off_queue) + f;
    L.scratch = b->ws + b->off_scr[f];
    L.scr_stride = b->scr_stride[f];
    uint32_t tail = 0;
    L.smem = form_smem(b, f, TT, &tail);
    L.tc_tail = tail;
    if (is_tc(f)) {
        L.MH = f == kFormTc128 ? 1 : 2;
        L.n_cta = std::min(b->num_sms, n_items);
    } else {
        L.RA = cand;
        const int occ = form_occupancy(f, cand, L.smem);
        L.n_cta = std::min(std::max(occ, 1) * b->num_sms, std::max(n_items, 1));
    }
    L.n_cta = std::min(L.n_cta, b->max_cta[f]);
    return L;
}

int launch_form(const BatchLaunch &L, int f, void *stream) {
    if (is_tc(f)) return launch_tc_batch(L, stream);
    return f == kFormF64 ? launch_simt_batch_f64(L, stream) : launch_simt_batch_f32(L, stream);
}

// Upload params and items for the shapes of candidate choice `ch` (per form),
// K_run grid points; returns, per form, the items' offset and count.
aqt_status upload(aqt_batch *b, const int ch[kForms], int K_run, std::vector<int> &TT, std::vector<int> &tiles,
                  size_t item_off[kForms], int n_items[kForms]) {
    TT.assign(b->mem.size(), 0);
    tiles.assign(b->mem.size(), 0);
    std::vector<BatchItem> all;
    for (int f = 0; f < kForms; ++f) {
        item_off[f] = all.size();
        n_items[f] = 0;
        if (b->members[f].empty()) continue;
        if (!shapes_for(b, f, ch[f], TT, tiles)) return bfail(b, AQT_EINVAL, "no tile shape fits the batch");
        auto it = form_items(b, f, TT, tiles);
        n_items[f] = (int)it.size();
        all.insert(all.end(), it.begin(), it.end());
    }
    if (all.size() > b->n_items_max) return bfail(b, AQT_EINVAL, "internal: batch item table too small");
    auto ps = member_params(b, TT, tiles, K_run);
    cudaError_t e = cudaMemcpy(b->ws + b->off_params, ps.data(), ps.size() * sizeof(RunParams), cudaMemcpyHostToDevice);
    if (!e && !all.empty())
        e = cudaMemcpy(b->ws + b->off_items, all.data(), all.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
    if (e) return bcuda(b, e, "batch parameter upload");
    return AQT_OK;
}

// Zero the counters of every member and the queues, on `st`.
cudaError_t reset_counters(aqt_batch *b, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (auto &m : b->mem) {
        if (!e) e = cudaMemsetAsync(m.p.jcount, 0, 8, st);
        if (!e) e = cudaMemsetAsync(m.p.status, 0, 4, st);
        if (!e && m.p.norm_err) e = cudaMemsetAsync(m.p.norm_err, 0, 4, st);
    }
    if (!e) e = cudaMemsetAsync(b->ws + b->off_queue, 0, 4 * kForms, st);
    return e;
}

aqt_status check_members(aqt_batch *b) {
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (ctx_version(b->ctx[i]) != b->mem[i].version)
            return bfail(b, AQT_EINVAL,
                         "member " + std::to_string(i) + " changed (inputs, tables or workspace) after the batch was created");
    return AQT_OK;
}

// Time every candidate of every form on the batch itself (first kTuneSteps
// grid points), keep the fastest; cached per signature.
aqt_status tune(aqt_batch *b) {
    cudaError_t e = cudaSetDevice(b->device);
    if (e) return bcuda(b, e, "cudaSetDevice");
    for (int f = 0; f < kForms; ++f) {
        if (b->members[f].empty()) continue;
        const std::string sig = signature(b, f);
        {
            std::lock_guard<std::mutex> lk(g_cache_mu);
            auto it = g_tune_cache.find(sig);
            if (it != g_tune_cache.end()) {
                b->chosen[f] = it->second;
                continue;
            }
        }
        float best = 0.0f;
        int best_c = -1;
        for (int c : b->cands[f]) {
            int ch[kForms] = {-1, -1, -1, -1};
            for (int g = 0; g < kForms; ++g) ch[g] = b->cands[g].empty() ? -1 : b->cands[g][0];
            ch[f] = c;
            std::vector<int> TT, tiles;
            size_t ioff[kForms];
            int nit[kForms];
            {
                std::vector<int> t1(b->mem.size()), t2(b->mem.size());
                if (!shapes_for(b, f, c, t1, t2)) continue;
            }
            aqt_status s = upload(b, ch, kTuneSteps, TT, tiles, ioff, nit);
            if (s != AQT_OK) return s;
            const BatchLaunch L = form_launch(b, f, c, TT, ioff[f], nit[f]);
            float ms = 0.0f;
            for (int rep = 0; rep < 2; ++rep) {  // the first run warms the caches and sets the attributes
                e = reset_counters(b, b->cap);
                if (!e) e = cudaEventRecord(b->ev0, b->cap);
                if (!e) e = (cudaError_t)launch_form(L, f, b->cap);
                if (!e) e = cudaEventRecord(b->ev1, b->cap);
                if (!e) e = cudaEventSynchronize(b->ev1);
                if (!e) e = cudaEventElapsedTime(&ms, b->ev0, b->ev1);
                if (e) return bcuda(b, e, "batch tuning run");
            }
            if (best_c < 0 || ms < best) {
                best = ms;
                best_c = c;
            }
        }
        if (best_c < 0) return bfail(b, AQT_EINVAL, "no tile shape fits the batch");
        b->chosen[f] = best_c;
        std::lock_guard<std::mutex> lk(g_cache_mu);
        g_tune_cache[sig] = best_c;
    }
    b->tuned = true;
    return AQT_OK;
}

void drop_graph(aqt_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Final shapes on the device, and the graph of one run: counters zeroed, one
// persistent launch per form, the observable reduction.
aqt_status build_graph(aqt_batch *b) {
    drop_graph(b);
    std::vector<int> TT, tiles;
    size_t ioff[kForms];
    int nit[kForms];
    aqt_status s = upload(b, b->chosen, 0, TT, tiles, ioff, nit);
    if (s != AQT_OK) return s;
    b->TT = TT;
    b->n_tiles = tiles;
    BatchLaunch L[kForms];
    for (int f = 0; f < kForms; ++f) {
        if (b->members[f].empty()) continue;
        L[f] = form_launch(b, f, b->chosen[f], TT, ioff[f], nit[f]);
        L[f].prepare_only = true;  // kernel attributes are set outside the capture
        const int ce = launch_form(L[f], f, b->cap);
        if (ce) return bcuda(b, (cudaError_t)ce, "batch kernel attributes");
        L[f].prepare_only = false;
    }
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e) return bcuda(b, e, "cudaStreamBeginCapture");
    e = reset_counters(b, b->cap);
    for (int f = 0; f < kForms && !e; ++f)
        if (!b->members[f].empty()) e = (cudaError_t)launch_form(L[f], f, b->cap);
    if (!e)
        e = (cudaError_t)launch_reduce_batch(reinterpret_cast<const RunParams *>(b->ws + b->off_params),
                                             (int)b->mem.size(), b->max_K, b->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (!e) e = e2;
    if (e) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, e, "batch graph capture");
    }
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e) {
        drop_graph(b);
        return bcuda(b, e, "cudaGraphInstantiate");
    }
    return AQT_OK;
}

}  // namespace

extern "C" {

aqt_status aqt_batch_create(aqt_batch **out, aqt_ctx *const *members, int n_members) {
    if (!out) return AQT_EINVAL;
    *out = nullptr;
    if (!members || n_members < 1) return AQT_EINVAL;
    aqt_batch *b = new (std::nothrow) aqt_batch();
    if (!b) return AQT_EINVAL;
    for (int i = 0; i < n_members; ++i) {
        if (!members[i]) {
            delete b;
            return AQT_EINVAL;
        }
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) {
                delete b;
                return AQT_EINVAL;  // a context's outputs can belong to one member only
            }
        BatchMember m;
        aqt_status s = batch_member(members[i], &m);
        if (s != AQT_OK) {
            delete b;
            return s;
        }
        if (i > 0 && m.device != b->device) {
            delete b;
            return AQT_EINVAL;
        }
        b->device = m.device;
        b->num_sms = m.num_sms;
        b->ctx.push_back(members[i]);
        b->mem.push_back(m);
        b->form.push_back(form_of(m));
        b->members[b->form.back()].push_back(i);
        b->max_K = std::max(b->max_K, m.p.K);
    }
    // candidates: SIMT rows per thread (every member must fit), tensor-core tile caps
    for (int f = 0; f < kForms; ++f) {
        if (b->members[f].empty()) continue;
        if (is_tc(f)) {
            // the largest tile the shared and tensor memory take (tc_shape from 256 per SM down)
            const int cap = tc_shape(f == kFormTc128 ? 128 : 256, 256, 1);
            b->cands[f].push_back(cap);
            const int half = ((cap / 2) + 7) & ~7;
            if (half >= 16 && half < cap) b->cands[f].push_back(half);
        } else {
            for (int ra : {4, 2, 8}) {
                std::vector<int> t1(b->mem.size()), t2(b->mem.size());
                if (shapes_for(b, f, ra, t1, t2)) b->cands[f].push_back(ra);
            }
            if (b->cands[f].empty()) {
                delete b;
                return AQT_EINVAL;
            }
        }
        b->chosen[f] = b->cands[f][0];
    }
    cudaError_t e = cudaSetDevice(b->device);
    if (!e) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreate(&b->ev0);
    if (!e) e = cudaEventCreate(&b->ev1);
    if (e) {
        if (b->cap) cudaStreamDestroy(b->cap);
        if (b->ev0) cudaEventDestroy(b->ev0);
        if (b->ev1) cudaEventDestroy(b->ev1);
        delete b;
        return AQT_ECUDA;
    }
    // workspace layout: sized for the largest candidate footprint
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    b->off_params = take(b->mem.size() * sizeof(RunParams));
    b->off_queue = take(4 * kForms);
    size_t items = 0;
    b->off_obs.assign(b->mem.size(), 0);
    std::vector<size_t> obs_need(b->mem.size(), 0);
    for (int f = 0; f < kForms; ++f) {
        if (b->members[f].empty()) continue;
        size_t items_f = 0;
        int n_max = 0, tt_max = 8;
        for (int c : b->cands[f]) {
            std::vector<int> TT(b->mem.size()), tiles(b->mem.size());
            if (!shapes_for(b, f, c, TT, tiles)) continue;
            size_t it = 0;
            for (int i : b->members[f]) {
                it += tiles[i];
                obs_need[i] = std::max(obs_need[i], (size_t)tiles[i] * b->mem[i].p.K * 24);
                tt_max = std::max(tt_max, TT[i]);
            }
            items_f = std::max(items_f, it);
        }
        for (int i : b->members[f]) n_max = std::max(n_max, b->mem[i].p.N);
        items += items_f;
        if (is_tc(f)) {
            b->max_cta[f] = b->num_sms;
            b->scr_stride[f] = tc_batch_scratch_double2(n_max, tt_max);
        } else {
            b->max_cta[f] = kMaxSimtCtaPerSm * b->num_sms;
            b->scr_stride[f] = (size_t)kScratchSlots * kSlotDouble2 * n_max;
        }
    }
    b->n_items_max = items;
    b->off_items = take(items * sizeof(BatchItem));
    for (size_t i = 0; i < b->mem.size(); ++i) b->off_obs[i] = take(obs_need[i]);
    for (int f = 0; f < kForms; ++f)
        if (!b->members[f].empty()) b->off_scr[f] = take((size_t)b->max_cta[f] * b->scr_stride[f] * 16);
    b->need = off;
    *out = b;
    return AQT_OK;
}

void aqt_batch_destroy(aqt_batch *b) {
    if (!b) return;
    if (b->device >= 0) cudaSetDevice(b->device);
    drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
}

const char *aqt_batch_last_error(const aqt_batch *b) { return b ? b->err.c_str() : "null batch"; }

aqt_status aqt_batch_workspace_size(aqt_batch *b, size_t *bytes) {
    if (!b || !bytes) return AQT_EINVAL;
    *bytes = b->need;
    return AQT_OK;
}

aqt_status aqt_batch_bind_workspace(aqt_batch *b, void *dptr, size_t bytes) {
    if (!b) return AQT_EINVAL;
    if (!dptr || ((uintptr_t)dptr & 255)) return bfail(b, AQT_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < b->need) return bfail(b, AQT_ENOMEM, "workspace smaller than aqt_batch_workspace_size");
    drop_graph(b);
    b->ws = (unsigned char *)dptr;
    b->ws_bytes = bytes;
    return AQT_OK;
}

aqt_status aqt_batch_tune(aqt_batch *b, void *stream) {
    if (!b) return AQT_EINVAL;
    if (!b->ws) return bfail(b, AQT_EINVAL, "bind a workspace before tuning");
    aqt_status s = check_members(b);
    if (s != AQT_OK) return s;
    // order the tuning runs after the caller's pending work on `stream`
    cudaError_t e = cudaSetDevice(b->device);
    if (!e) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e) return bcuda(b, e, "stream synchronize");
    s = tune(b);
    if (s != AQT_OK) return s;
    drop_graph(b);
    return AQT_OK;
}

aqt_status aqt_batch_run(aqt_batch *b, void *stream) {
    if (!b) return AQT_EINVAL;
    if (!b->ws) return bfail(b, AQT_EINVAL, "bind a workspace before running");
    aqt_status s = check_members(b);
    if (s != AQT_OK) return s;
    cudaError_t e = cudaSetDevice(b->device);
    if (e) return bcuda(b, e, "cudaSetDevice");
    if (!b->tuned) {
        e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e) return bcuda(b, e, "stream synchronize");
        s = tune(b);
        if (s != AQT_OK) return s;
    }
    if (!b->exec) {
        s = build_graph(b);
        if (s != AQT_OK) return s;
    }
    e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e) return bcuda(b, e, "cudaGraphLaunch");
    for (aqt_ctx *c : b->ctx) batch_member_ran(c, stream);
    return AQT_OK;
}

aqt_status aqt_batch_sync(aqt_batch *b, int32_t *member_status) {
    if (!b) return AQT_EINVAL;
    aqt_status worst = AQT_OK;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        const aqt_status s = aqt_sync(b->ctx[i]);
        if (member_status) member_status[i] = (int32_t)s;
        if (s != AQT_OK && (worst == AQT_OK || worst == AQT_EOVERFLOW)) {
            worst = s;
            b->err = "member " + std::to_string(i) + ": " + aqt_last_error(b->ctx[i]);
        }
    }
    return worst;
}

aqt_status aqt_batch_get_shape(aqt_batch *b, int member, int32_t *shape) {
    if (!b || !shape || member < 0 || member >= (int)b->mem.size()) return AQT_EINVAL;
    if (b->TT.empty()) return bfail(b, AQT_EINVAL, "run the batch first");
    const int f = b->form[member];
    shape[0] = is_tc(f) ? 2 : f;
    shape[1] = b->TT[member];
    shape[2] = is_tc(f) ? (f == kFormTc128 ? 1 : 2) : b->chosen[f];
    shape[3] = b->n_tiles[member];
    return AQT_OK;
}

}  // extern "C"
