// Several systems stepped together, and the launch-shape autotuner.
//
// A batch holds contexts of systems of any sizes, each with its own stream and
// workspace.  One leapfrog step of every system is captured once into a single
// CUDA graph: a fork on the batch's stream, each system's kernels as a branch on
// its own stream, a join.  Every batch step is then one cudaGraphLaunch; the
// device-side step counters advance inside the graph.  The dominant work, the
// walker-side tensor-core contraction's GEMM-Z, runs for all systems that use it
// (one operand arithmetic, Y images in one chunk of walkers) in one persistent
// launch on the batch's stream: each branch runs up to the contraction's images,
// the branches join, contract_tcw_kernel takes every system's blocks from one
// list, and the branches fork again for the rest of the step.
//
// The autotuner times the candidate launch shapes of the heaviest kernels on a
// context's own data (warps per block of the overlap kernel, pairs per block of
// the tensor-core contraction, threads per block of the trial-orbital kernel)
// and keeps the fastest; choices are cached per problem shape for the process.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "kernels.cuh"

using namespace afq;

struct afqmc_batch {
    int n;
    std::vector<afqmc_ctx*> ctxs;
    cudaStream_t root;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaEvent_t fork, zdone;
    std::vector<cudaEvent_t> joins, pre;
    long long kernels_per_step;   // kernel nodes in the graph
    int shared_z;                 // systems whose GEMM-Z runs in the batch's one persistent launch
};

// Operand arithmetic of the walker-side contraction (0 bf16x3, 1 fp16x3, 2 fp16x6),
// or -1 when the context does not use that form with one chunk of walkers.
static int shared_z_mode(const afqmc_ctx* c) {
    if (c->cfg.precision == AFQMC_PRECISION_FP64 || tc_kind(&c->cfg) != 5) return -1;
    const int mode = c->cfg.precision == AFQMC_PRECISION_FP16X6 ? 2 : (c->cfg.precision == AFQMC_PRECISION_FP16X3 ? 1 : 0);
    return contract_tcw_single_chunk(c->d, mode) ? mode : -1;
}

#define BK(call)                                                                                            \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return set_error(AFQMC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

typedef std::tuple<int, int, int, int, int, int, int> TuneKey;
static std::mutex g_tune_mu;
static std::map<TuneKey, std::tuple<int, int, int>> g_tune_cache;

template <class F>
static afqmc_status time_ms(cudaStream_t s, F launch, int reps, float* out) {
    cudaEvent_t a, b;
    BK(cudaEventCreate(&a));
    BK(cudaEventCreate(&b));
    BK(launch());   // warm-up (module load, attributes)
    BK(cudaEventRecord(a, s));
    for (int r = 0; r < reps; ++r) BK(launch());
    BK(cudaEventRecord(b, s));
    BK(cudaEventSynchronize(b));
    float ms = 0.f;
    BK(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *out = ms / reps;
    return AFQMC_OK;
}

extern "C" afqmc_status afqmc_autotune(afqmc_ctx* ctx, int* chosen) {
    if (!ctx) return set_error(AFQMC_ERR_ARG, "ctx is NULL");
    Dims& d = ctx->d;
    const afqmc_config& c = ctx->cfg;
    TuneKey key(d.N, d.nu, d.nd, d.G, d.W, d.P, c.precision);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            d.ov_wpb = std::get<0>(it->second);
            d.tc_tp = std::get<1>(it->second);
            d.cheb_threads = std::get<2>(it->second);
            if (chosen) { chosen[0] = d.ov_wpb; chosen[1] = d.tc_tp; chosen[2] = d.cheb_threads; }
            return AFQMC_OK;
        }
    }
    Workspace& w = ctx->ws;
    cudaStream_t s = ctx->stream;
    const int reps = 3;
    afqmc_status st;
    // overlap kernel: matrices per block
    int best_wpb = 4;
    float best = 1e30f;
    for (int wpb : {1, 2, 4}) {
        Dims t = d;
        t.ov_wpb = wpb;
        float ms;
        st = time_ms(s, [&] { return overlap_lu(s, t, 0, w.Phi, phi_stride(t), w.phi, w.logdet, w.Theta, nullptr,
                                                w.status, t.pairs, t.P); }, reps, &ms);
        if (st != AFQMC_OK) return st;
        if (ms < best) { best = ms; best_wpb = wpb; }
    }
    d.ov_wpb = best_wpb;
    // tensor-core contraction: pairs per block (largest that fits, and smaller)
    int best_tp = 0;
    if (c.precision != AFQMC_PRECISION_FP64 && tc_kind(&c) != 5) {   // the general walker-side form has no tuned shape
        const bool f16 = c.precision == AFQMC_PRECISION_FP16X3;
        const int ovl = tc_kind(&c) == 2 ? OVL_TRIAL : OVL_THETA;
        for (int spin = 0; spin < 2; ++spin)
            BK(overlap_lu(s, d, spin, w.Phi, phi_stride(d), w.phi, w.logdet, w.Theta, nullptr, w.status, d.pairs,
                          d.P, ovl));
        best = 1e30f;
        for (int tp : {0, 4, 2, 1}) {
            Dims t = d;
            t.tc_tp = tp;
            float ms;
            st = time_ms(s, [&] { return contract_tc(s, t, w.Lt, w.Phi, w.Theta, w.phi, w.Yimg, w.vpair, w.epair, w.status, f16); }, 1,
                         &ms);
            if (st != AFQMC_OK) return st;
            if (ms < best) { best = ms; best_tp = tp; }
        }
    }
    d.tc_tp = best_tp;
    // trial orbitals: threads per block
    int best_th = 256;
    best = 1e30f;
    for (int th : {128, 256}) {
        float ms;
        st = time_ms(s, [&] {
            return c.precision == AFQMC_PRECISION_FP64
                       ? trial_orbitals(s, d.N, d.nu, d.pairs, w.Sprop, w.Phi0, w.Phiprop, w.alive, d.P, w.status, th)
                       : trial_orbitals_df(s, d.N, d.nu, d.pairs, w.Sprop, w.Phi0, w.Phiprop, w.alive, d.P, w.status, th,
                                           trial_orbitals_df_supported(d.N, d.nu) ||
                                               trial_orbitals_dfg_supported(d.N, d.nu));
        }, 1, &ms);
        if (st != AFQMC_OK) return st;
        if (ms < best) { best = ms; best_th = th; }
    }
    d.cheb_threads = best_th;
    ctx->measured = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = std::make_tuple(d.ov_wpb, d.tc_tp, d.cheb_threads);
    }
    if (chosen) { chosen[0] = d.ov_wpb; chosen[1] = d.tc_tp; chosen[2] = d.cheb_threads; }
    return AFQMC_OK;
}

extern "C" afqmc_status afqmc_batch_create(int n, afqmc_ctx* const* ctxs, void* stream, afqmc_batch** out) {
    if (!out || n < 1 || !ctxs) return set_error(AFQMC_ERR_ARG, "bad arguments");
    *out = nullptr;
    cudaStream_t root = (cudaStream_t)stream;
    if (!root) return set_error(AFQMC_ERR_ARG, "the batch needs a non-default stream");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return set_error(AFQMC_ERR_ARG, "context %d is NULL", i);
        if (!ctxs[i]->stream || ctxs[i]->stream == root)
            return set_error(AFQMC_ERR_ARG, "context %d needs its own non-default stream", i);
        if (ctxs[i]->profiling) return set_error(AFQMC_ERR_ARG, "context %d is profiling", i);
    }
    afqmc_batch* b = new afqmc_batch();
    b->n = n;
    b->ctxs.assign(ctxs, ctxs + n);
    b->root = root;
    b->graph = nullptr;
    b->exec = nullptr;
    b->fork = b->zdone = nullptr;
    b->joins.assign(n, nullptr);
    b->pre.assign(n, nullptr);
    // the systems whose GEMM-Z shares one launch: those of the first such system's arithmetic
    int zmode = -1;
    std::vector<char> shared(n, 0);
    TcwZMulti zm;
    zm.n = 0;
    zm.first[0] = 0;
    for (int i = 0; i < n; ++i) {
        const int md = shared_z_mode(ctxs[i]);
        if (md < 0 || (zmode >= 0 && md != zmode) || zm.n + 2 > TCWZ_MAXWORK) continue;
        TcwZArgs a[2];
        bool ok = true;
        for (int q = 0; q < 2 && ok; ++q) ok = contract_tcw_zargs(ctxs[i]->d, ctxs[i]->ws.tcw, ctxs[i]->ws.status, md, q, &a[q]);
        if (!ok) continue;
        zmode = md;
        shared[i] = 1;
        for (int q = 0; q < 2; ++q) {
            if (a[q].n == 0) continue;
            zm.a[zm.n] = a[q];
            zm.first[zm.n + 1] = zm.first[zm.n] + a[q].blocks;
            ++zm.n;
        }
    }
    b->shared_z = 0;
    for (int i = 0; i < n; ++i) b->shared_z += shared[i];
    afqmc_status st = AFQMC_OK;
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->zdone, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->pre[i], cudaEventDisableTiming);
    // the contexts' earlier work must be done before the capture
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamSynchronize(ctxs[i]->stream);
    const long long launches_before = afqmc_launch_count();
    if (e == cudaSuccess) e = cudaStreamBeginCapture(root, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        cudaError_t e2 = cudaEventRecord(b->fork, root);
        if (b->shared_z > 0) {
            // the sharing systems up to their images; then GEMM-Z of all of them in one
            // launch; then their steps' remainder and the other systems' whole steps
            for (int i = 0; i < n && e2 == cudaSuccess && st == AFQMC_OK; ++i) {
                if (!shared[i]) continue;
                e2 = cudaStreamWaitEvent(ctxs[i]->stream, b->fork, 0);
                if (e2 == cudaSuccess) st = batch_step_part(ctxs[i], 1);
                if (e2 == cudaSuccess && st == AFQMC_OK) e2 = cudaEventRecord(b->pre[i], ctxs[i]->stream);
                if (e2 == cudaSuccess && st == AFQMC_OK) e2 = cudaStreamWaitEvent(root, b->pre[i], 0);
            }
            if (e2 == cudaSuccess && st == AFQMC_OK) e2 = contract_tcw_multi(root, zm, zmode, ctxs[0]->d.wait_polls);
            if (e2 == cudaSuccess && st == AFQMC_OK) e2 = cudaEventRecord(b->zdone, root);
        }
        for (int i = 0; i < n && e2 == cudaSuccess && st == AFQMC_OK; ++i) {
            e2 = cudaStreamWaitEvent(ctxs[i]->stream, shared[i] ? b->zdone : b->fork, 0);
            if (e2 == cudaSuccess) {
                if (shared[i]) {
                    st = batch_step_part(ctxs[i], 2);
                    ctxs[i]->steps_taken -= 1;   // captured, not run
                } else {
                    st = afqmc_step(ctxs[i], 1);
                    ctxs[i]->steps_taken -= 1;   // captured, not run
                }
            }
            if (e2 == cudaSuccess && st == AFQMC_OK) e2 = cudaEventRecord(b->joins[i], ctxs[i]->stream);
            if (e2 == cudaSuccess && st == AFQMC_OK) e2 = cudaStreamWaitEvent(root, b->joins[i], 0);
        }
        cudaError_t e3 = cudaStreamEndCapture(root, &b->graph);
        e = e2 != cudaSuccess ? e2 : e3;
    }
    // captured kernels are counted when the graph runs, not now
    b->kernels_per_step = afqmc_launch_count() - launches_before;
    count_launches(-b->kernels_per_step);
    if (e == cudaSuccess && st == AFQMC_OK) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess || st != AFQMC_OK) {
        if (st == AFQMC_OK) st = set_error(AFQMC_ERR_CUDA, "capturing the batch step: %s", cudaGetErrorString(e));
        afqmc_batch_destroy(b);
        return st;
    }
    *out = b;
    return AFQMC_OK;
}

extern "C" afqmc_status afqmc_batch_step(afqmc_batch* b, int n_steps) {
    if (!b || n_steps < 0) return set_error(AFQMC_ERR_ARG, "bad arguments");
    for (int k = 0; k < n_steps; ++k) {
        cudaError_t e = cudaGraphLaunch(b->exec, b->root);
        if (e != cudaSuccess) return set_error(AFQMC_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
        count_launches(b->kernels_per_step);
    }
    for (afqmc_ctx* c : b->ctxs) {
        c->steps_taken += n_steps;
        c->measured = false;
    }
    return AFQMC_OK;
}

extern "C" int afqmc_batch_shared_contractions(const afqmc_batch* b) { return b ? b->shared_z : -1; }

extern "C" afqmc_status afqmc_batch_sync(afqmc_batch* b) {
    if (!b) return set_error(AFQMC_ERR_ARG, "bad arguments");
    BK(cudaStreamSynchronize(b->root));
    return AFQMC_OK;
}

extern "C" void afqmc_batch_destroy(afqmc_batch* b) {
    if (!b) return;
    if (b->root) cudaStreamSynchronize(b->root);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->zdone) cudaEventDestroy(b->zdone);
    for (cudaEvent_t e : b->joins)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->pre)
        if (e) cudaEventDestroy(e);
    delete b;
}
