// C ABI of the library (declared in include/afqmc.h): configuration checks,
// the workspace layout, and the order of kernels in init, step and measure.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <map>
#include <algorithm>
#include <mutex>
#include <utility>

#include "kernels.cuh"

using namespace afq;

static thread_local char g_err[512] = "";

static afqmc_status fail(afqmc_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

afqmc_status set_error(afqmc_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(AFQMC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" const char* afqmc_last_error(void) { return g_err; }
static std::atomic<long long> g_launches{0};
void afq::count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

extern "C" int64_t afqmc_launch_count(void) { return g_launches.load(); }

// A trial other than the real one-slice form (complex alpha, or several slices).
static bool general_trial(const afqmc_config* c) {
    return c->trial_alpha_im != 0.0 || c->trial_alpha_re != 1.0 || c->trial_slices > 1;
}

extern "C" int afqmc_contract_kernel(const afqmc_config* cfg) {
    if (!cfg) return -1;
    if (cfg->precision == AFQMC_PRECISION_FP64) {
        if (general_trial(cfg)) return contract_fp64c_supported(cfg->N, cfg->n_up, cfg->n_dn) ? 6 : -1;
        if (cfg->rcache) return contract_fp64r_supported(cfg->N, cfg->n_up, cfg->n_dn) ? 4 : -1;
        if (contract_fp64_walker_side(cfg->N, cfg->n_up, cfg->n_dn, cfg->n_paths)) return 3;
        return contract_fp64_supported(cfg->N, cfg->n_up, cfg->n_dn) ? 0 : -1;
    }
    return tc_kind(cfg);
}

// operand arithmetic of the walker-side tensor-core form: 0 bf16x3, 1 fp16x3, 2 fp16x6
static int tc_mode(const afqmc_config* c) {
    return c->precision == AFQMC_PRECISION_FP16X6 ? 2 : (c->precision == AFQMC_PRECISION_FP16X3 ? 1 : 0);
}

int tc_kind(const afqmc_config* c) {
    const bool f16 = c->precision == AFQMC_PRECISION_FP16X3;
    const bool tcw = contract_tcw_supported(c->N, c->n_up, c->n_dn, c->n_chol, c->n_walkers, c->n_paths, tc_mode(c));
    // complex or multi-slice trial samples: the walker-side form, whose per-pair
    // operand B_p = conj(Phi_p) A_p^-T is complex for a real trial already
    if (general_trial(c)) return c->tc_form != AFQMC_TC_PER_PAIR && tcw ? 5 : -1;
    if (c->precision == AFQMC_PRECISION_FP16X6) {   // the walker-side form only
        if (c->tc_form == AFQMC_TC_PER_PAIR) return -1;
        return tcw ? 5 : -1;
    }
    const bool tc = contract_tc_supported(c->N, c->n_up, c->n_dn, f16);
    if (c->tc_form == AFQMC_TC_PER_PAIR) return tc ? 1 : -1;
    if (c->tc_form == AFQMC_TC_WALKER) return tcw ? 5 : -1;
    if (contract_tc_walker_side(c->N, c->n_up, c->n_dn, f16)) return 2;
    if (tc) return 1;
    return tcw ? 5 : -1;
}

// The mixed path's overlaps form A = Phi^T phi (and, for the walker-side contraction, B =
// Phi A^-T) in double-float: the general walker-side form with a real trial (at most 64
// electrons per spin, its limit).  The LU, log det and A^-1 stay FP64.
static bool overlaps_in_df(const afqmc_config* c) {
    return c->precision != AFQMC_PRECISION_FP64 && !general_trial(c) && c->n_up <= 64 && c->n_dn <= 64 &&
           tc_kind(c) == 5;
}

// The overlap matrices of the double-float path formed on the tensor cores (overlap_tc).
static bool overlaps_on_tc(const afqmc_config* c) {
    return overlaps_in_df(c) && c->overlap_form == AFQMC_OVERLAP_AUTO && overlap_tc_supported(c->N, c->n_up) &&
           (c->n_dn == 0 || overlap_tc_supported(c->N, c->n_dn));
}

// The proposal matrices S formed on the tensor cores (sprop_tc): for the tensor-core
// trial orbitals only, whose digits of S' carry the same precision.
static bool s_on_tc_cfg(const afqmc_config* c) {
    const int f = c->trial_form;
    return c->precision != AFQMC_PRECISION_FP64 && !general_trial(c) && f != AFQMC_TRIAL_DF &&
           trial_orbitals_tc_supported(c->N, c->n_up) && (f == AFQMC_TRIAL_TC || c->N > 64) &&
           sprop_tc_supported(c->K, (long long)c->N * c->N);
}

// Double-float copies of `doubles` FP64 values (u_to_df).
static cudaError_t df_copy(cudaStream_t s, const void* src, long long doubles, void* dst) {
    return u_to_df(s, doubles, static_cast<const double*>(src), dst);
}

static std::mutex g_smem_mu;
static std::map<std::pair<const void*, int>, size_t> g_smem_limit;   // (kernel, device) -> bytes allowed

cudaError_t afq::raise_smem_limit(const void* kernel, size_t bytes) {
    if (bytes == 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_smem_mu);
    size_t& cur = g_smem_limit[std::make_pair(kernel, dev)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// ---------------------------------------------------------------- phase profiling
// While enabled, afqmc_step records a CUDA event on the context's stream at
// every phase boundary; afqmc_profile_read converts consecutive pairs into
// per-phase milliseconds.  Recording events does not synchronise the stream.
static long long g_mark_launches = 0;

static afqmc_status prof_flush(afqmc_ctx* ctx) {
    if (ctx->prof_used == 0) return AFQMC_OK;
    CK(cudaEventSynchronize(ctx->prof_events[ctx->prof_used - 1]));
    for (int i = 1; i < ctx->prof_used; ++i) {
        int ph = ctx->prof_phase[i];
        if (ph < 0) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->prof_events[i - 1], ctx->prof_events[i]));
        ctx->prof_ms[ph] += ms;
    }
    ctx->prof_used = 0;
    return AFQMC_OK;
}

// phase >= 0: the phase that ends here; phase < 0: a step starts here.
static afqmc_status prof_mark(afqmc_ctx* ctx, int phase) {
    if (!ctx->profiling) return AFQMC_OK;
    long long now = g_launches.load();
    if (phase >= 0) ctx->prof_launches[phase] += now - g_mark_launches;
    g_mark_launches = now;
    if (ctx->prof_used == ctx->prof_cap) {
        afqmc_status st = prof_flush(ctx);
        if (st != AFQMC_OK) return st;
        if (phase >= 0) {   // keep the boundary: re-record the start of this phase is lost, so restart at a step mark
            phase = -1;
        }
    }
    CK(cudaEventRecord(ctx->prof_events[ctx->prof_used], ctx->stream));
    ctx->prof_phase[ctx->prof_used] = phase;
    ctx->prof_used++;
    return AFQMC_OK;
}

extern "C" afqmc_status afqmc_profile(afqmc_ctx* ctx, int enable) {
    if (!ctx) return fail(AFQMC_ERR_ARG, "ctx is NULL");
    if (enable && !ctx->prof_events) {
        ctx->prof_cap = 256 * (PH_COUNT + 1);
        ctx->prof_events = (cudaEvent_t*)calloc(ctx->prof_cap, sizeof(cudaEvent_t));
        ctx->prof_phase = (int*)calloc(ctx->prof_cap, sizeof(int));
        if (!ctx->prof_events || !ctx->prof_phase) return fail(AFQMC_ERR_ARG, "out of host memory");
        for (int i = 0; i < ctx->prof_cap; ++i) CK(cudaEventCreate(&ctx->prof_events[i]));
    }
    if (!enable) {
        afqmc_status st = prof_flush(ctx);
        if (st != AFQMC_OK) return st;
    }
    ctx->profiling = enable != 0;
    return AFQMC_OK;
}

extern "C" afqmc_status afqmc_profile_read(afqmc_ctx* ctx, double* out, int len) {
    if (!ctx || !out || len < 0) return fail(AFQMC_ERR_ARG, "bad arguments");
    afqmc_status st = prof_flush(ctx);
    if (st != AFQMC_OK) return st;
    for (int i = 0; i < len; ++i) {
        double v = 0.0;
        if (i < PH_COUNT) v = ctx->prof_ms[i];
        else if (i < 2 * PH_COUNT) v = (double)ctx->prof_launches[i - PH_COUNT];
        else if (i == 2 * PH_COUNT) v = (double)ctx->prof_steps;
        out[i] = v;
    }
    for (int i = 0; i < PH_COUNT; ++i) { ctx->prof_ms[i] = 0.0; ctx->prof_launches[i] = 0; }
    ctx->prof_steps = 0;
    return AFQMC_OK;
}


extern "C" void afqmc_config_default(afqmc_config* c) {
    memset(c, 0, sizeof *c);
    c->n_sweeps = 1;
    c->n_burn = 20;
    c->constraint = AFQMC_CONSTRAINT_COMBINED;
    c->proposal = AFQMC_PROPOSAL_PRIOR;
    c->precision = AFQMC_PRECISION_FP64;
    c->taylor_order = 6;
    c->history_capacity = 1024;
    c->pcn_beta = 1.0;
    c->kill_threshold = 1e-10;
    c->rw_step = 0.3;
    c->mlp_mix = 0.1;
    c->mlp_lr = 1e-3;
    c->mlp_train = 0;
    c->refine_tol = 1e-4;
    c->trial_alpha_re = 1.0;
    c->trial_alpha_im = 0.0;
    c->trial_slices = 1;
}

// The tensor-core contraction's pairs with the largest error get recomputed in
// FP64 (refine.cu): mixed precision, the per-pair form (it keeps Theta), and a
// positive per-walker tolerance.
static bool refine_enabled(const afqmc_config* c) {
    if (c->precision == AFQMC_PRECISION_FP64 || !(c->refine_tol > 0.0)) return false;
    const int k = tc_kind(c);
    return (k == 1 || k == 5) && contract_fp64_supported(c->N, c->n_up, c->n_dn);
}

static const char* check_config(const afqmc_config* c) {
    if (!c) return "config is NULL";
    if (c->N < 1 || c->N > 256) return "N must be in [1, 256]";
    if (c->n_up < 1 || c->n_up > c->N || c->n_up > 64) return "n_up must be in [1, min(N, 64)]";
    if (c->n_dn < 0 || c->n_dn > c->n_up) return "n_dn must be in [0, n_up]";
    if (c->n_chol < 1 || c->K < 1) return "n_chol and K must be >= 1";
    if (c->n_walkers < 1 || c->n_paths < 1 || c->n_paths > 1024) return "n_walkers >= 1 and 1 <= n_paths <= 1024";
    if ((long long)c->n_walkers * c->n_paths > (1ll << 31)) return "too many walker-path pairs";
    if (c->n_sweeps < 1 || c->n_burn < 0) return "n_sweeps >= 1 and n_burn >= 0";
    if (c->constraint < 0 || c->constraint > 2) return "unknown constraint";
    if (c->proposal < 0 || c->proposal > 3) return "unknown proposal";
    if ((c->proposal == AFQMC_PROPOSAL_RW || c->proposal == AFQMC_PROPOSAL_MLP) && !(c->rw_step > 0.0))
        return "rw_step must be > 0";
    if (c->proposal == AFQMC_PROPOSAL_MLP && !(c->mlp_mix >= 0.0 && c->mlp_mix <= 1.0)) return "mlp_mix in [0, 1]";
    if (c->proposal == AFQMC_PROPOSAL_MLP && !(c->mlp_lr >= 0.0)) return "mlp_lr must be >= 0";
    if (c->precision < AFQMC_PRECISION_FP64 || c->precision > AFQMC_PRECISION_FP16X6) return "unknown precision";
    if (c->taylor_order < 1 || c->taylor_order > 32) return "taylor_order must be in [1, 32]";
    if (c->history_capacity < 1) return "history_capacity must be >= 1";
    if (!(c->dtau > 0.0)) return "dtau must be > 0";
    if (c->proposal == AFQMC_PROPOSAL_PCN && !(c->pcn_beta > 0.0 && c->pcn_beta <= 1.0)) return "pcn_beta in (0, 1]";
    if (!(c->kill_threshold >= 0.0)) return "kill_threshold must be >= 0";
    if (!(c->refine_tol >= 0.0)) return "refine_tol must be >= 0";
    if (c->importance < AFQMC_IMPORTANCE_HYBRID || c->importance > AFQMC_IMPORTANCE_LOCAL_ENERGY)
        return "unknown importance function";
    if (c->pop_period < 0) return "pop_period must be >= 0";
    if (c->pop_period > 0 && c->n_walkers > 65535) return "population control supports at most 65535 walkers";
    if (c->rcache != 0 && c->rcache != 1) return "rcache must be 0 or 1";
    if (c->wait_polls < 0 || c->wait_polls > (1ll << 31)) return "wait_polls must be in [0, 2^31]";
    if (c->trial_form < AFQMC_TRIAL_AUTO || c->trial_form > AFQMC_TRIAL_TC) return "unknown trial_form";
    if (c->overlap_form < AFQMC_OVERLAP_AUTO || c->overlap_form > AFQMC_OVERLAP_DF) return "unknown overlap_form";
    if (c->rcache && c->precision != AFQMC_PRECISION_FP64) return "rcache needs precision FP64";
    if (c->rcache && !contract_fp64r_supported(c->N, c->n_up, c->n_dn))
        return "sizes too large for the cached half-rotation form (Theta and one matrix per warp, 4 warps per block)";
    if (c->walker_offset < 0 || (c->walker_offset + c->n_walkers) * (long long)c->n_paths > (1ll << 32))
        return "walker_offset out of range of the 32-bit stream entity";
    if (c->precision == AFQMC_PRECISION_FP64 && !contract_fp64_supported(c->N, c->n_up, c->n_dn))
        return "sizes too large for the FP64 contraction kernel";
    if (c->tc_form < AFQMC_TC_AUTO || c->tc_form > AFQMC_TC_WALKER) return "unknown tc_form";
    if (c->trial_slices < 1 || c->trial_slices > 8) return "trial_slices must be in [1, 8]";
    if (!isfinite(c->trial_alpha_re) || !isfinite(c->trial_alpha_im) ||
        (c->trial_alpha_re == 0.0 && c->trial_alpha_im == 0.0))
        return "trial alpha must be finite and non-zero";
    if (general_trial(c)) {
        if (c->proposal == AFQMC_PROPOSAL_MLP)
            return "the learned proposal is defined for the one-slice real trial only";
        if (c->rcache) return "complex or multi-slice trials need rcache = 0";
        if (!trial_orbitals_c_supported(c->N, c->n_up) || !contract_fp64c_supported(c->N, c->n_up, c->n_dn))
            return "sizes too large for the complex trial-orbital or contraction kernels";
        if ((long long)c->K * c->trial_slices > 4096) return "too many hidden variables per sample";
    }
    if (c->precision != AFQMC_PRECISION_FP64 && tc_kind(c) < 0)
        return "sizes not supported by the chosen tensor-core contraction (per-pair form: N <= 128, n_up <= 32; "
               "walker-side form: N <= 256, n_up <= 64)";
    if (3ull * c->N * c->n_up * 8 > 200 * 1024)
        return "sizes too large for the trial-orbital kernel (3 N n_up doubles of shared memory)";
    return nullptr;
}

static Dims dims_of(const afqmc_config* c) {
    Dims d{};   // value-initialised: launch shapes at their defaults
    d.N = c->N; d.nu = c->n_up; d.nd = c->n_dn; d.nt = c->n_up + c->n_dn;
    d.G = c->n_chol; d.K = c->K; d.W = c->n_walkers; d.P = c->n_paths;
    d.pairs = (long long)c->n_walkers * c->n_paths;
    d.ov_wpb = 0;
    d.tc_tp = 0;
    d.cheb_threads = 0;
    if (c->wait_polls > 0) d.wait_polls = (uint32_t)c->wait_polls;
    d.KU = c->K;
    if (general_trial(c)) {   // complex storage of Phi; K counts the variables of every slice
        d.cphi = 1;
        d.slices = c->trial_slices;
        d.K = c->K * c->trial_slices;
    }
    return d;
}

// Carve the workspace into 256-byte aligned buffers; with base == nullptr
// only the total is computed.
static size_t layout(const afqmc_config* c, char* base, Workspace* ws) {
    Dims d = dims_of(c);
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        off = (off + 255) & ~(size_t)255;
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    size_t N = d.N, NN = N * N, nt = d.nt, nu = d.nu, G = d.G, K = d.K, W = d.W, pairs = d.pairs;
    Workspace w{};
    // h and the L_g back to back: [h; L_1; ...; L_G] is one (G+1) N x N matrix
    w.h = (double*)take((G + 1) * NN * 8);
    w.L = w.h + NN;
    w.Phi0 = (double*)take(N * nu * 8);
    w.U = (double*)take((size_t)d.KU * NN * 8);
    w.Pslice = d.slices > 1 ? (double*)take(NN * 8) : nullptr;
    w.Vtmp = d.slices > 1 ? (double2*)take(pairs * N * nu * 16) : nullptr;
    w.Udf = c->precision != AFQMC_PRECISION_FP64 ? take(K * NN * 8) : nullptr;
    w.T = (double*)take(NN * 8);
    w.expT = (double*)take(NN * 8);
    // the double-float propagation needs its work arrays in shared memory
    const bool prop_df = c->precision != AFQMC_PRECISION_FP64 && propagate_in_smem(d.N, d.nt);
    w.Ldf = prop_df || refine_enabled(c) ? take(G * NN * 8) : nullptr;
    w.hdf = refine_enabled(c) ? take(NN * 8) : nullptr;
    w.xdf = c->precision != AFQMC_PRECISION_FP64 ? take(std::max(pairs * K, 2 * W * G) * 8) : nullptr;
    w.expTdf = prop_df ? take(NN * 8) : nullptr;
    w.scratchNN = (double*)take(3 * NN * 8);
    const int tck = c->precision != AFQMC_PRECISION_FP64 ? tc_kind(c) : -1;
    const bool f16c = c->precision == AFQMC_PRECISION_FP16X3;
    w.Lt = (tck == 1 || tck == 2) ? take(contract_tc_image_bytes(d.N, d.nu, d.nd, d.G, f16c)) : nullptr;
    w.Yimg = tck == 2 ? take(contract_tcy_yimage_bytes(d.N, d.nu, d.nd, d.G, d.W, f16c)) : nullptr;
    w.tcw = tck == 5 ? take(contract_tcw_work_bytes(d.N, d.nu, d.nd, d.G, d.W, d.P, tc_mode(c))) : nullptr;
    const size_t ywalk = c->precision == AFQMC_PRECISION_FP64 ? contract_fp64_walker_bytes(d.N, d.nu, d.nd, d.G, d.W, d.P)
                                                              : 0;
    w.ywalk = ywalk ? take(ywalk) : nullptr;
    w.phi = (double2*)take(W * N * nt * 16);
    w.weight = (double*)take(W * 8);
    w.x = (double*)take(pairs * K * 8);
    w.Phi = (double*)take(pairs * phi_stride(d) * 8);
    w.logdet = (double2*)take(pairs * 2 * 16);
    w.logov = (double2*)take(pairs * 16);
    w.Theta = (double2*)take(pairs * N * nt * 16);
    w.vpair = (double2*)take(pairs * G * 16);
    w.epair = (double2*)take(pairs * 16);
    w.logdet_new = (double2*)take(pairs * 2 * 16);
    w.logov_cur = (double2*)take(pairs * 16);
    w.sumS = (double2*)take(W * 16);
    w.vbar = (double2*)take(W * G * 16);
    w.ebar = (double2*)take(W * 16);
    w.y = (double2*)take(W * G * 16);
    w.logshift = (double2*)take(W * 16);
    const bool refine = refine_enabled(c);
    w.refine_th2 = refine ? (double*)take(2 * pairs * 8) : nullptr;   // per pair (and spin)
    w.refine_items = refine ? (int*)take(pairs * 4) : nullptr;
    w.refine_n = refine ? (int*)take(4) : nullptr;
    w.refine_lam = refine ? (double*)take((G + 1) * 8) : nullptr;
    w.Aplanes = (double*)take(2 * W * NN * 8);
    w.phi_new = (double2*)take(W * N * nt * 16);
    w.propbuf = propagate_in_smem(d.N, d.nt) ? nullptr : (double2*)take(W * 2 * N * nt * 16);
    w.old_sum = (double2*)take(W * 16);
    w.ratio = (double2*)take(W * 16);
    w.Iabs = (double*)take(W * 8);
    w.alive = (int*)take(W * 4);
    if (c->pop_period > 0) {
        w.comb_cum = (double*)take(W * 8);
        w.comb_hit = (int*)take(W * 4);
        w.comb_slot = (int*)take(W * 4);
        w.comb_from = (int*)take(W * 4);
        w.comb_flag = (int*)take(2 * 4);
    }
    w.xsave = (double*)take(pairs * K * 8);
    w.Phisave = (double*)take(pairs * phi_stride(d) * 8);
    w.msum0 = (double2*)take(W * 16);
    w.macc = (double2*)take(2 * W * 16);
    w.mout = (double2*)take((2 * W + 2) * 16);
    if (c->rcache) {
        w.rc = (double*)take(rcache_bytes(c->N, c->n_up, c->n_chol, (long long)c->n_walkers * c->n_paths));
        w.rdirty = (int*)take(pairs * 4);
        w.rlist = (int*)take(pairs * 4);
        w.rcount = (int*)take(4);
    }
    w.xprop = (double*)take(pairs * K * 8);
    w.Sprop = (double*)take(pairs * NN * 8);
    w.Phiprop = (double*)take(pairs * phi_stride(d) * 8);
    if (c->precision != AFQMC_PRECISION_FP64) {
        w.cheb_redo = (int*)take((pairs + 1) * 4);   // list, then its count at [pairs]
    }
    if (overlaps_in_df(c)) {
        w.Phidf = take(pairs * phi_stride(d) * 8);
        w.phidf = take(W * N * nt * 16);
    }
    if (overlaps_on_tc(c)) w.Aov = take(pairs * ((size_t)c->n_up * c->n_up + (size_t)c->n_dn * c->n_dn) * 16);
    if (s_on_tc_cfg(c)) w.Uimg = take(sprop_u_image_bytes(c->K, (long long)c->N * c->N));
    w.logdet_prop = (double2*)take(pairs * 2 * 16);
    w.history = (double*)take((size_t)c->history_capacity * 4 * 8);
    w.reduce = (double*)take(8 * 8);
    w.counters = (unsigned long long*)take(16 * 8);
    w.status = (int*)take(4);
    if (c->proposal == AFQMC_PROPOSAL_MLP) {
        MlpBuffers& m = w.mlp;
        const size_t H = 256, Kp = (K + 15) / 16 * 16, Wp = (W + 15) / 16 * 16, np = (size_t)mlp_n_params(d.K);
        m.Kp = (int)Kp;
        m.Wp = (int)Wp;
        m.UPhi0 = (double*)take(K * N * nu * 8);
        m.Theta0 = (double2*)take(W * N * nt * 16);
        m.logdet0 = (double2*)take(W * 2 * 16);
        m.featf = (float*)take(Wp * Kp * 4);
        m.featb = (__nv_bfloat16*)take(Wp * Kp * 2);
        m.theta = (float*)take(np * 4);
        m.adam_m = (float*)take(np * 4);
        m.adam_v = (float*)take(np * 4);
        m.grad = (float*)take(np * 4);
        m.W1b = (__nv_bfloat16*)take(H * Kp * 2);
        m.W2b = (__nv_bfloat16*)take(H * H * 2);
        m.W3b = (__nv_bfloat16*)take(2 * Kp * H * 2);
        m.Zf = (float*)take(Wp * H * 4);
        m.H1f = (float*)take(Wp * H * 4);
        m.H2f = (float*)take(Wp * H * 4);
        m.dHf = (float*)take(Wp * H * 4);
        m.dZf = (float*)take(Wp * H * 4);
        m.H1b = (__nv_bfloat16*)take(Wp * H * 2);
        m.H2b = (__nv_bfloat16*)take(Wp * H * 2);
        m.dZb = (__nv_bfloat16*)take(Wp * H * 2);
        m.outf = (float*)take(Wp * 2 * Kp * 4);
        m.doutf = (float*)take(Wp * 2 * Kp * 4);
        m.doutb = (__nv_bfloat16*)take(Wp * 2 * Kp * 2);
        m.mu = (float*)take(W * K * 4);
        m.logv = (float*)take(W * K * 4);
        m.logv_raw = (float*)take(W * K * 4);
        m.gW1p = (float*)take(H * Kp * 4);
        m.gb1 = (float*)take(H * 4);
        m.gW2 = (float*)take(H * H * 4);
        m.gb2 = (float*)take(H * 4);
        m.gW3p = (float*)take(2 * Kp * H * 4);
        m.gb3p = (float*)take(2 * Kp * 4);
        m.loss_part = (double*)take(W * 8);
        m.loss = (double*)take(8);
        m.counter = (unsigned long long*)take(8);
        m.status = w.status;
    }
    w.total = (off + 255) & ~(size_t)255;
    if (ws) *ws = w;
    return w.total;
}

extern "C" size_t afqmc_workspace_bytes(const afqmc_config* cfg) {
    if (check_config(cfg)) return 0;
    return layout(cfg, nullptr, nullptr);
}

static StepParams params_of(const afqmc_config* c) {
    StepParams p;
    p.seed = c->seed; p.woff = c->walker_offset; p.dtau = c->dtau; p.pcn_beta = c->pcn_beta; p.e_shift = c->e_shift;
    p.rw_step = c->rw_step; p.mlp_mix = c->mlp_mix;
    p.kill_threshold = c->kill_threshold; p.constraint = c->constraint; p.proposal = c->proposal;
    p.taylor_order = c->taylor_order; p.history_capacity = c->history_capacity;
    p.importance = c->importance; p.pop_period = c->pop_period;
    return p;
}

// The mixed-precision path forms S and the trial orbitals in double-float
// arithmetic (S stored as double-float pairs) when the trial kernel's vectors fit
// its shared memory (S there too, or read from global memory); the FP64 path in FP64.
static bool s_in_df(const afqmc_ctx* ctx) {
    return ctx->cfg.precision != AFQMC_PRECISION_FP64 &&
           (trial_orbitals_df_supported(ctx->d.N, ctx->d.nu) || trial_orbitals_dfg_supported(ctx->d.N, ctx->d.nu));
}

// Trial orbitals of the mixed-precision path on the tensor cores (trial_tc.cu).
static bool trial_on_tc(const afqmc_ctx* ctx) {
    const int f = ctx->cfg.trial_form;
    return ctx->cfg.precision != AFQMC_PRECISION_FP64 && f != AFQMC_TRIAL_DF &&
           trial_orbitals_tc_supported(ctx->d.N, ctx->d.nu) && (f == AFQMC_TRIAL_TC || ctx->d.N > 64);
}

// S_m = sum_k X[m, k] U_k into ws.Sprop for `M` rows of X.
static cudaError_t form_S(afqmc_ctx* ctx, const double* X, long long M) {
    const Dims& d = ctx->d;
    Workspace& w = ctx->ws;
    const long long NN = (long long)d.N * d.N;
    if (w.Uimg && trial_on_tc(ctx) && s_in_df(ctx))
        return sprop_tc(ctx->stream, M, d.K, NN, X, w.Uimg, w.Sprop, w.status, d.wait_polls);
    if (s_in_df(ctx)) return gemm_df(ctx->stream, (int)M, (int)NN, d.K, X, w.Udf, w.Sprop, w.xdf);
    gemm_nn_f64(ctx->stream, (int)M, (int)NN, d.K, 1.0, X, d.K, w.U, NN, 0.0, w.Sprop, NN);
    return cudaGetLastError();
}

// Trial orbitals exp(S) Phi0 for `problems` matrices S in ws.Sprop: FP64 on the
// FP64 path, double-float arithmetic on the mixed-precision path.
static cudaError_t trial_orbitals_of(afqmc_ctx* ctx, long long problems, double* Out, const int* alive, int P) {
    const Dims& d = ctx->d;
    Workspace& w = ctx->ws;
    if (ctx->cfg.precision == AFQMC_PRECISION_FP64)
        return trial_orbitals(ctx->stream, d.N, d.nu, problems, w.Sprop, w.Phi0, Out, alive, P, w.status, d.cheb_threads);
    if (trial_on_tc(ctx))
        return trial_orbitals_tc(ctx->stream, d.N, d.nu, problems, w.Sprop, s_in_df(ctx), w.Phi0, Out, alive, P, w.status,
                                 w.cheb_redo, w.cheb_redo + d.pairs, w.counters, d.wait_polls);
    return trial_orbitals_df(ctx->stream, d.N, d.nu, problems, w.Sprop, w.Phi0, Out, alive, P, w.status, d.cheb_threads,
                             s_in_df(ctx));
}

// Trial orbitals Phi(x) of `problems` rows of X (the proposal or path variables):
// S = sum_k x_k U_k and exp(S) Phi0, or, for a complex or multi-slice trial, the
// chain exp(alpha S_m) P ... P exp(alpha S_1) Phi0 with S_l from the l-th block of
// K variables (complex output).
static cudaError_t trial_samples(afqmc_ctx* ctx, const double* X, long long problems, double* Out, const int* alive,
                                 int P) {
    const Dims& d = ctx->d;
    Workspace& w = ctx->ws;
    if (!d.cphi) {
        cudaError_t e = form_S(ctx, X, problems);
        return e != cudaSuccess ? e : trial_orbitals_of(ctx, problems, Out, alive, P);
    }
    const long long NN = (long long)d.N * d.N;
    const double2 alpha = cmk(ctx->cfg.trial_alpha_re, ctx->cfg.trial_alpha_im);
    double2* O = reinterpret_cast<double2*>(Out);
    for (int l = 0; l < d.slices; ++l) {
        gemm_nn_f64(ctx->stream, (int)problems, (int)NN, d.KU, 1.0, X + (size_t)l * d.KU, d.K, w.U, NN, 0.0, w.Sprop,
                    NN);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (l == 0) {
            e = trial_orbitals_c(ctx->stream, d.N, d.nu, problems, w.Sprop, alpha, w.Phi0, nullptr, O, alive, P, w.status);
        } else {
            e = slice_propagate(ctx->stream, d.N, d.nu, problems, w.Pslice, O, w.Vtmp, alive, P);
            if (e == cudaSuccess)
                e = trial_orbitals_c(ctx->stream, d.N, d.nu, problems, w.Sprop, alpha, nullptr, w.Vtmp, O, alive, P,
                                     w.status);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One Metropolis sweep of every path against the walker orbitals `orbitals`
// (phi' during a step, phi during burn-in).
static afqmc_status mcmc_sweep(afqmc_ctx* ctx, const double2* orbitals, uint32_t tag_prop, uint32_t tag_acc,
                               uint32_t sweep, bool burn_in = false) {
    const Dims& d = ctx->d;
    Workspace& w = ctx->ws;
    cudaStream_t s = ctx->stream;
    StepParams p = params_of(&ctx->cfg);
    if (burn_in && p.proposal == AFQMC_PROPOSAL_MLP) p.proposal = AFQMC_PROPOSAL_PRIOR;   // no network output yet
    afqmc_status st;
    CK(propose(s, d, p, w.counters, tag_prop, tag_acc, sweep, w.x, w.alive, w.mlp.mu, w.mlp.logv, w.xprop));
    if (!d.cphi) CK(form_S(ctx, w.xprop, d.pairs));
    if ((st = prof_mark(ctx, PH_PROPOSE)) != AFQMC_OK) return st;
    if (d.cphi)
        CK(trial_samples(ctx, w.xprop, d.pairs, w.Phiprop, w.alive, d.P));
    else
        CK(trial_orbitals_of(ctx, d.pairs, w.Phiprop, w.alive, d.P));
    if ((st = prof_mark(ctx, PH_TRIAL)) != AFQMC_OK) return st;
    if (w.Phidf) {
        CK(df_copy(s, w.Phiprop, d.pairs * phi_stride(d), w.Phidf));
        CK(df_copy(s, orbitals, d.W * (long long)d.N * d.nt * 2, w.phidf));
    }
    if (w.Aov) CK(overlap_tc(s, d, w.Phidf, phi_stride(d), w.phidf, w.alive, w.Aov, w.status));
    CK(overlap_lu_both(s, d, w.Phiprop, phi_stride(d), orbitals, w.logdet_prop, nullptr, w.alive, w.status,
                       d.pairs, d.P, OVL_THETA, nullptr, w.Phidf, w.phidf, false, w.Aov));
    if ((st = prof_mark(ctx, PH_MCMC_OVERLAP)) != AFQMC_OK) return st;
    CK(accept(s, d, p, w.counters, tag_acc, sweep, w.logdet_prop, w.xprop, w.Phiprop, w.alive, w.mlp.mu, w.mlp.logv,
              w.logov_cur, w.x, w.Phi, w.counters, w.rdirty));
    return prof_mark(ctx, PH_ACCEPT);
}

// Local energies, force-bias values and path signs at the current walkers,
// and the mixed-estimator sums into ws.reduce[0..2].
// part 0: the whole measurement.  For a batch that runs the walker-side
// contraction's GEMM-Z of all its systems in one launch: part 1 stops after the
// contraction's images, part 2 starts with its per-pair finish (the batch runs
// GEMM-Z in between; the context's Y images then fit one chunk of walkers).
static afqmc_status measure(afqmc_ctx* ctx, int part = 0) {
    const Dims& d = ctx->d;
    Workspace& w = ctx->ws;
    cudaStream_t s = ctx->stream;
    afqmc_status st;
    const bool f16 = ctx->cfg.precision == AFQMC_PRECISION_FP16X3;
    const bool fp64 = ctx->cfg.precision == AFQMC_PRECISION_FP64;
    const int tck = fp64 ? -1 : tc_kind(&ctx->cfg);
    const int ovl = fp64 ? (!w.rc && !d.cphi && contract_fp64_walker_side(d.N, d.nu, d.nd, d.P) ? OVL_INVERSE : OVL_THETA)
                         : (tck == 2 || tck == 5 ? OVL_TRIAL : OVL_THETA);
    if (part == 2) {
        CK(contract_tcw_finish(s, d, w.tcw, w.vpair, w.epair, tc_mode(&ctx->cfg)));
    } else {
    if (w.Phidf) {
        CK(df_copy(s, w.Phi, d.pairs * phi_stride(d), w.Phidf));
        CK(df_copy(s, w.phi, d.W * (long long)d.N * d.nt * 2, w.phidf));
    }
    if (w.Aov) CK(overlap_tc(s, d, w.Phidf, phi_stride(d), w.phidf, nullptr, w.Aov, w.status));
    CK(overlap_lu_both(s, d, w.Phi, phi_stride(d), w.phi, w.logdet, w.Theta, nullptr, w.status, d.pairs, d.P,
                       ovl, tck == 5 && w.refine_items ? w.refine_th2 : nullptr, w.Phidf, w.phidf,
                       w.Phidf && ovl == OVL_TRIAL, w.Aov));
    if ((st = prof_mark(ctx, PH_OVERLAP)) != AFQMC_OK) return st;
    if (part == 1) {
        if (tck != 5) return fail(AFQMC_ERR_ARG, "a split measurement needs the walker-side contraction");
        CK(contract_tcw_images(s, d, w.tcw, w.Theta, w.phi, w.status, tc_mode(&ctx->cfg), w.Phidf != nullptr));
        return AFQMC_OK;
    }
    if (ctx->cfg.precision != AFQMC_PRECISION_FP64) {
        if (tck == 5)
            CK(contract_tcw(s, d, w.tcw, w.Theta, w.phi, w.vpair, w.epair, w.status, tc_mode(&ctx->cfg),
                            w.Phidf != nullptr));
        else
            CK(contract_tc(s, d, w.Lt, w.Phi, w.Theta, w.phi, w.Yimg, w.vpair, w.epair, w.status, f16));
    } else if (w.rc) {   // cached half-rotated matrices, refreshed for the paths that moved
        CK(rcache_refresh(s, d, w.h, w.Phi, w.rdirty, w.rlist, w.rcount, w.rc, w.counters));
        CK(contract_fp64r(s, d, w.rc, w.Theta, w.vpair, w.epair));
    } else if (ovl == OVL_INVERSE)
        CK(contract_fp64_walker(s, d, w.h, w.L, w.Phi, w.Theta, w.phi, w.ywalk, w.vpair, w.epair));
    else
        CK(d.cphi ? contract_fp64c(s, d, w.h, w.L, reinterpret_cast<const double2*>(w.Phi), w.Theta, w.vpair, w.epair)
                  : contract_fp64(s, d, w.h, w.L, w.Phi, w.Theta, w.vpair, w.epair, d.pairs));
    }
    if ((st = prof_mark(ctx, PH_CONTRACT)) != AFQMC_OK) return st;
    if (w.refine_items && tck == 5) {
        // the pairs whose error would put their walker above refine_tol, again: selected
        // by ||A_p^-1||_F^2 from the overlap kernel with the per-pair form's error model
        // (measured per-pair errors of this form sit at 0.3-0.5 of it for N = 120 and 200),
        // their Theta formed in place of B, then the double-float per-pair contraction;
        // the log-overlaps go to scratch
        // unit roundoff of the model: fp16x3 and bf16x3 operands about 20 bits; fp16x6 operands about
        // 31 bits, the entries reaching the traces as FP32 numbers (24 bits)
        const double u = tc_mode(&ctx->cfg) == 2 ? 0x1p-24 : 0x1p-20;
        CK(refine_select(s, d, ctx->cfg.refine_tol, w.refine_lam + d.G, w.logdet, w.Theta, w.refine_th2, w.alive,
                         w.refine_items, w.refine_n, w.counters, w.refine_th2, u));
        for (int spin = 0; spin < 2; ++spin)
            CK(overlap_lu(s, d, spin, w.Phi, phi_stride(d), w.phi, w.logdet_new, w.Theta, nullptr, w.status, d.pairs,
                          d.P, OVL_THETA, nullptr, w.refine_items, w.refine_n));
        if (d.cphi)   // complex trial samples: the listed pairs in FP64
            CK(contract_fp64c(s, d, w.h, w.L, reinterpret_cast<const double2*>(w.Phi), w.Theta, w.vpair, w.epair,
                              w.refine_items, w.refine_n));
        else
            CK(contract_fp64_listed(s, d, w.h, w.L, w.Phi, w.Theta, w.vpair, w.epair, w.refine_items, w.refine_n,
                                    d.pairs, w.hdf, w.Ldf, w.refine_th2, d.pairs));
    } else if (w.refine_items) {   // per-pair form: Theta is at hand
        CK(refine_select(s, d, ctx->cfg.refine_tol, w.refine_lam + d.G, w.logdet, w.Theta, w.refine_th2, w.alive,
                         w.refine_items, w.refine_n, w.counters));
        CK(contract_fp64_listed(s, d, w.h, w.L, w.Phi, w.Theta, w.vpair, w.epair, w.refine_items, w.refine_n, d.pairs,
                                w.hdf, w.Ldf, w.refine_th2, d.pairs));
    }
    if ((st = prof_mark(ctx, PH_REFINE)) != AFQMC_OK) return st;
    CK(walker_average(s, d, w.logdet, w.vpair, w.epair, w.logov, w.sumS, w.vbar, w.ebar));
    CK(energy_reduce(s, d, w.weight, w.ebar, w.sumS, w.reduce));
    return prof_mark(ctx, PH_AVERAGE);
}

extern "C" afqmc_status afqmc_init(const afqmc_config* cfg, const double* h, const double* L, const double* Phi0,
                                   const double* U, void* workspace, size_t workspace_bytes, void* stream,
                                   afqmc_ctx** out) {
    return afqmc_init_trial(cfg, h, L, Phi0, U, nullptr, workspace, workspace_bytes, stream, out);
}

extern "C" afqmc_status afqmc_init_trial(const afqmc_config* cfg, const double* h, const double* L,
                                         const double* Phi0, const double* U, const double* slice_prop,
                                         void* workspace, size_t workspace_bytes, void* stream, afqmc_ctx** out) {
    if (!out) return fail(AFQMC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (const char* m = check_config(cfg)) return fail(AFQMC_ERR_ARG, "%s", m);
    if (!h || !L || !Phi0 || !U) return fail(AFQMC_ERR_ARG, "h, L, Phi0 and U must not be NULL");
    if (cfg->trial_slices > 1 && !slice_prop)
        return fail(AFQMC_ERR_ARG, "a multi-slice trial needs the propagator between slices (afqmc_init_trial)");
    size_t need = layout(cfg, nullptr, nullptr);
    if (!workspace || workspace_bytes < need)
        return fail(AFQMC_ERR_WORKSPACE, "workspace needs %zu bytes, got %zu", need, workspace_bytes);
    if (((uintptr_t)workspace & 255) != 0) return fail(AFQMC_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(AFQMC_ERR_WORKSPACE, "workspace is not device memory");
    }
    afqmc_ctx* ctx = (afqmc_ctx*)calloc(1, sizeof(afqmc_ctx));
    if (!ctx) return fail(AFQMC_ERR_ARG, "out of host memory");
    ctx->cfg = *cfg;
    ctx->d = dims_of(cfg);
    ctx->stream = (cudaStream_t)stream;
    layout(cfg, (char*)workspace, &ctx->ws);
    afqmc_status st = AFQMC_OK;
    do {
        const Dims& d = ctx->d;
        Workspace& w = ctx->ws;
        cudaStream_t s = ctx->stream;
        size_t NN = (size_t)d.N * d.N;
        auto copy_in = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
            return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
        };
        cudaError_t e = copy_in(w.h, h, NN * 8);
        if (e == cudaSuccess) e = copy_in(w.L, L, (size_t)d.G * NN * 8);
        if (e == cudaSuccess) e = copy_in(w.Phi0, Phi0, (size_t)d.N * d.nu * 8);
        if (e == cudaSuccess) e = copy_in(w.U, U, (size_t)d.KU * NN * 8);
        if (e == cudaSuccess && w.Pslice) e = copy_in(w.Pslice, slice_prop, NN * 8);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.counters, 0, 16 * 8, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.status, 0, 4, s);
        if (e != cudaSuccess) { st = fail(AFQMC_ERR_CUDA, "copying inputs: %s", cudaGetErrorString(e)); break; }
        StepParams p = params_of(cfg);
        if (w.tcw && (e = contract_tcw_prepare(s, d, w.h, w.L, w.tcw, tc_mode(cfg))) !=
                         cudaSuccess) {
            st = fail(AFQMC_ERR_CUDA, "tensor-core operand image: %s", cudaGetErrorString(e));
            break;
        }
        if (w.Lt &&
            (e = contract_tc_prepare(s, d.N, d.nu, d.nd, d.G, w.h, w.L, w.Lt,
                                     cfg->precision == AFQMC_PRECISION_FP16X3)) != cudaSuccess) {
            st = fail(AFQMC_ERR_CUDA, "tensor-core operand image: %s", cudaGetErrorString(e));
            break;
        }
        if (w.refine_lam && (e = refine_scale(s, d.N, d.G, w.L, w.refine_lam, w.refine_lam + d.G)) != cudaSuccess) {
            st = fail(AFQMC_ERR_CUDA, "refinement scale: %s", cudaGetErrorString(e));
            break;
        }
        if ((e = one_body_propagator(s, d.N, d.G, cfg->dtau, w.h, w.L, w.T, w.scratchNN, w.expT)) != cudaSuccess) {
            st = fail(AFQMC_ERR_CUDA, "one-body propagator: %s", cudaGetErrorString(e));
            break;
        }
        // initial walkers phi_w = Phi(x_w), x_w ~ N(0, I), orthonormalised
        fill_normals(s, w.xprop, d.W, d.K, p.woff, p.seed, TAG_INIT_WALKER, w.counters, 0);
        if (w.Udf && ((e = u_to_df(s, (long long)d.K * NN, w.U, w.Udf)) != cudaSuccess ||
                      (w.Ldf && (e = u_to_df(s, (long long)d.G * NN, w.L, w.Ldf)) != cudaSuccess) ||
                      (w.hdf && (e = u_to_df(s, (long long)NN, w.h, w.hdf)) != cudaSuccess) ||
                      (w.expTdf && (e = u_to_df(s, (long long)NN, w.expT, w.expTdf)) != cudaSuccess))) {
            st = fail(AFQMC_ERR_CUDA, "double-float copies of U, L and exp(-tau T/2): %s", cudaGetErrorString(e));
            break;
        }
        if (w.Uimg && (e = sprop_u_images(s, d.K, NN, w.U, w.Uimg)) != cudaSuccess) {
            st = fail(AFQMC_ERR_CUDA, "digit images of U: %s", cudaGetErrorString(e));
            break;
        }
        if ((e = trial_samples(ctx, w.xprop, d.W, w.Phiprop, nullptr, 1)) != cudaSuccess) {
            st = fail(AFQMC_ERR_CUDA, "initial walkers: %s", cudaGetErrorString(e));
            break;
        }
        if (d.cphi)
            walkers_from_trial_c(s, d, reinterpret_cast<const double2*>(w.Phiprop), w.phi_new);
        else
            walkers_from_trial(s, d, w.Phiprop, w.phi_new);
        reorthonormalise(s, d, w.phi_new, w.phi, nullptr, w.status, d.W);
        // paths x_wp ~ N(0, I) and their orbitals
        fill_normals(s, w.x, d.pairs, d.K, p.woff * d.P, p.seed, TAG_INIT_PATH, w.counters, 0);
        if ((e = trial_samples(ctx, w.x, d.pairs, w.Phi, nullptr, d.P)) != cudaSuccess) {
            st = fail(AFQMC_ERR_CUDA, "initial paths: %s", cudaGetErrorString(e));
            break;
        }
        set_value(s, w.weight, d.W, 1.0);
        set_int(s, w.alive, d.W, 1);
        if (w.rdirty) set_int(s, w.rdirty, d.pairs, 1);   // nothing cached yet
        for (int spin = 0; spin < 2; ++spin)
            overlap_lu(s, d, spin, w.Phi, phi_stride(d), w.phi, w.logdet_new, nullptr, nullptr, w.status,
                       d.pairs, d.P);
        combine_logdet(s, d.pairs, w.logdet_new, w.logov_cur);
        if ((e = cudaGetLastError()) != cudaSuccess) { st = fail(AFQMC_ERR_CUDA, "init kernels: %s", cudaGetErrorString(e)); break; }
        if (cfg->proposal == AFQMC_PROPOSAL_MLP &&
            (e = mlp_prepare(s, d, w.mlp, w.U, w.Phi0, cfg->seed)) != cudaSuccess) {
            st = fail(AFQMC_ERR_CUDA, "learned proposal set-up: %s", cudaGetErrorString(e));
            break;
        }
        for (int b = 0; b < cfg->n_burn && st == AFQMC_OK; ++b)
            st = mcmc_sweep(ctx, w.phi, TAG_BURN_PROPOSE, TAG_BURN_ACCEPT, b, true);
        if (st != AFQMC_OK) break;
        // the burn-in acceptances are not counted in the run statistics
        if ((e = cudaMemsetAsync(w.counters, 0, 16 * 8, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            st = fail(AFQMC_ERR_CUDA, "init: %s", cudaGetErrorString(e));
            break;
        }
    } while (0);
    if (st != AFQMC_OK) {
        free(ctx);
        return st;
    }
    *out = ctx;
    return AFQMC_OK;
}

static afqmc_status step_rest(afqmc_ctx* ctx);

extern "C" afqmc_status afqmc_step(afqmc_ctx* ctx, int n_steps) {
    if (!ctx) return fail(AFQMC_ERR_ARG, "ctx is NULL");
    if (n_steps < 0) return fail(AFQMC_ERR_ARG, "n_steps must be >= 0");
    for (int it = 0; it < n_steps; ++it) {
        afqmc_status st = prof_mark(ctx, -1);
        if (st != AFQMC_OK) return st;
        if ((st = measure(ctx)) != AFQMC_OK) return st;      // Eq. (25)-(27), (16) at phi
        if ((st = step_rest(ctx)) != AFQMC_OK) return st;
    }
    ctx->measured = false;
    return AFQMC_OK;
}

// A step after its measurement: fields, propagation, ratios, Metropolis sweeps,
// hand-off, re-orthonormalisation, population control.
static afqmc_status step_rest(afqmc_ctx* ctx) {
    const Dims& d = ctx->d;
    Workspace& w = ctx->ws;
    cudaStream_t s = ctx->stream;
    StepParams p = params_of(&ctx->cfg);
    afqmc_status st;
    {
        CK(fields(s, d, p, w.counters, w.vbar, w.sumS, w.weight, w.alive, (double*)w.y, w.logshift));
        if (w.expTdf) {   // mixed precision: field planes and propagation in double-float
            CK(gemm_df(s, 2 * d.W, d.N * d.N, d.G, (const double*)w.y, w.Ldf, w.Aplanes, w.xdf));
        } else {
            gemm_nn_f64(s, 2 * d.W, d.N * d.N, d.G, 1.0, (const double*)w.y, d.G, w.L, (long long)d.N * d.N, 0.0,
                        w.Aplanes, (long long)d.N * d.N);
            CK(cudaGetLastError());
        }
        if ((st = prof_mark(ctx, PH_FIELDS)) != AFQMC_OK) return st;
        if (w.expTdf)
            CK(propagate_df(s, d, p, w.expTdf, w.Aplanes, w.phi, w.phi_new, w.alive));  // Eq. (12)
        else
            CK(propagate(s, d, p, w.expT, w.Aplanes, w.phi, w.phi_new, w.alive, w.propbuf));   // Eq. (12)
        if ((st = prof_mark(ctx, PH_PROPAGATE)) != AFQMC_OK) return st;
        if (w.Phidf) CK(df_copy(s, w.phi_new, d.W * (long long)d.N * d.nt * 2, w.phidf));   // Phi's copy: measure
        if (w.Aov) CK(overlap_tc(s, d, w.Phidf, phi_stride(d), w.phidf, w.alive, w.Aov, w.status));
        CK(overlap_lu_both(s, d, w.Phi, phi_stride(d), w.phi_new, w.logdet_new, nullptr, w.alive, w.status,
                           d.pairs, d.P, OVL_THETA, nullptr, w.Phidf, w.phidf, false, w.Aov));
        CK(ratios(s, d, w.logov, w.logdet_new, w.sumS, w.logshift, w.alive, w.logov_cur, w.old_sum, w.ratio, w.Iabs));
        if ((st = prof_mark(ctx, PH_RATIO)) != AFQMC_OK) return st;
        if (ctx->cfg.proposal == AFQMC_PROPOSAL_MLP) {       // proposal conditioned on the new walkers
            CK(mlp_features(s, d, w.mlp, w.Phi0, w.phi_new, w.status));
            CK(mlp_forward(s, d, w.mlp, d.W));
        }
        for (int m = 0; m < ctx->cfg.n_sweeps; ++m) {                                  // Eq. (23)
            st = mcmc_sweep(ctx, w.phi_new, TAG_PROPOSE, TAG_ACCEPT, (uint32_t)m);
            if (st != AFQMC_OK) return st;
        }
        if (ctx->cfg.proposal == AFQMC_PROPOSAL_MLP && ctx->cfg.mlp_train)   // one Adam step on the new states
            CK(mlp_backward(s, d, w.mlp, d.W, w.x, (float)ctx->cfg.mlp_lr, true));
        CK(handoff(s, d, p, w.logov_cur, w.old_sum, w.ratio, w.Iabs, w.ebar, w.alive, w.weight,
                   w.status));  // Eq. (28)-(29)
        CK(reorthonormalise(s, d, w.phi_new, w.phi, w.alive, w.status, d.W));
        CK(step_end(s, p, w.reduce, w.history, w.counters));
        if ((st = prof_mark(ctx, PH_FINISH)) != AFQMC_OK) return st;
        CK(population_control(s, d, p, w.counters, w.weight, w.phi, w.x, w.Phi, w.rc, w.rdirty, w.comb_cum, w.comb_hit,
                              w.comb_slot, w.comb_from, w.comb_flag));
        if ((st = prof_mark(ctx, PH_COMB)) != AFQMC_OK) return st;
        if (ctx->profiling) ctx->prof_steps++;
        ctx->steps_taken++;
    }
    return AFQMC_OK;
}

// One step of a batch whose walker-side GEMM-Z runs outside (part 1: up to the
// contraction's images; part 2: from its finish to the end of the step).
afqmc_status afq::batch_step_part(afqmc_ctx* ctx, int part) {
    if (part == 1) return measure(ctx, 1);
    afqmc_status st = measure(ctx, 2);
    if (st != AFQMC_OK) return st;
    if ((st = step_rest(ctx)) != AFQMC_OK) return st;
    ctx->measured = false;
    return AFQMC_OK;
}

// The device status word as a return value: a wait that timed out outranks the
// numerical flags (that measurement is not valid at all).
static afqmc_status status_result(int status) {
    if (status & STATUS_TIMEOUT)
        return fail(AFQMC_ERR_TIMEOUT, "device status word 0x%x: a tensor-core kernel gave up a bounded wait "
                                       "(4 timeout; 1 singular overlap, 2 non-finite value)", status);
    if (status)
        return fail(AFQMC_ERR_NUMERIC, "device status word 0x%x (1 singular overlap, 2 non-finite value)", status);
    return AFQMC_OK;
}

static afqmc_status read_status(afqmc_ctx* ctx, int* status) {
    CK(cudaMemcpyAsync(status, ctx->ws.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return AFQMC_OK;
}

extern "C" afqmc_status afqmc_energy(afqmc_ctx* ctx, double* e_mix, double* sum_w, double* mean_sign,
                                     double* e_walker) {
    if (!ctx) return fail(AFQMC_ERR_ARG, "ctx is NULL");
    afqmc_status st = measure(ctx);
    if (st != AFQMC_OK) return st;
    double r[3];
    CK(cudaMemcpyAsync(r, ctx->ws.reduce, sizeof r, cudaMemcpyDeviceToHost, ctx->stream));
    if (e_walker)
        CK(cudaMemcpyAsync(e_walker, ctx->ws.ebar, (size_t)ctx->d.W * 16, cudaMemcpyDeviceToHost, ctx->stream));
    int status = 0;
    if ((st = read_status(ctx, &status)) != AFQMC_OK) return st;
    ctx->measured = true;
    if (e_mix) *e_mix = r[1] > 0 ? r[0] / r[1] : 0.0;
    if (sum_w) *sum_w = r[1];
    if (mean_sign) *mean_sign = r[1] > 0 ? r[2] / r[1] : 0.0;
    return status_result(status);
}

extern "C" afqmc_status afqmc_trial_orbitals(afqmc_ctx* ctx, const double* x, int64_t n, double* out) {
    if (!ctx || !x || !out || n < 0) return fail(AFQMC_ERR_ARG, "bad arguments");
    const Dims& d = ctx->d;
    if (n > d.pairs) return fail(AFQMC_ERR_ARG, "n = %lld exceeds n_walkers * n_paths = %lld", (long long)n, d.pairs);
    if (n == 0) return AFQMC_OK;
    Workspace& w = ctx->ws;
    CK(cudaMemcpyAsync(w.xprop, x, (size_t)n * d.K * 8, cudaMemcpyDefault, ctx->stream));
    CK(trial_samples(ctx, w.xprop, n, w.Phiprop, nullptr, 1));
    CK(cudaMemcpyAsync(out, w.Phiprop, (size_t)n * phi_stride(d) * 8, cudaMemcpyDefault, ctx->stream));
    int status = 0;
    afqmc_status st = read_status(ctx, &status);
    return st != AFQMC_OK ? st : status_result(status);
}

extern "C" afqmc_status afqmc_observables(afqmc_ctx* ctx, double* logov, double* e_local, double* force_bias) {
    if (!ctx) return fail(AFQMC_ERR_ARG, "ctx is NULL");
    if (!ctx->measured) return fail(AFQMC_ERR_ARG, "call afqmc_energy first");
    const Dims& d = ctx->d;
    if (logov) CK(cudaMemcpyAsync(logov, ctx->ws.logov, d.pairs * 16, cudaMemcpyDeviceToHost, ctx->stream));
    if (e_local) CK(cudaMemcpyAsync(e_local, ctx->ws.epair, d.pairs * 16, cudaMemcpyDeviceToHost, ctx->stream));
    if (force_bias)
        CK(cudaMemcpyAsync(force_bias, ctx->ws.vbar, (size_t)d.W * d.G * 16, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return AFQMC_OK;
}

extern "C" afqmc_status afqmc_history(afqmc_ctx* ctx, double* out, int n, int* n_out) {
    if (!ctx || !out || n < 0) return fail(AFQMC_ERR_ARG, "bad arguments");
    int cap = ctx->cfg.history_capacity;
    long long taken = ctx->steps_taken;
    long long k = n;
    if (k > taken) k = taken;
    if (k > cap) k = cap;
    for (long long i = 0; i < k; ++i) {
        long long st = taken - k + i;
        CK(cudaMemcpyAsync(out + 4 * i, ctx->ws.history + 4 * (st % cap), 32, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    if (n_out) *n_out = (int)k;
    return AFQMC_OK;
}

__global__ void weight_stats_kernel(int W, const double* __restrict__ weight, double* out4) {
    __shared__ double smin[256], smax[256], ssum[256], slive[256];
    double mn = INFINITY, mx = -INFINITY, sm = 0.0, lv = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        double v = weight[w];
        mn = fmin(mn, v); mx = fmax(mx, v); sm += v; lv += (v > 0.0);
    }
    smin[threadIdx.x] = mn; smax[threadIdx.x] = mx; ssum[threadIdx.x] = sm; slive[threadIdx.x] = lv;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + off]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + off]);
            ssum[threadIdx.x] += ssum[threadIdx.x + off];
            slive[threadIdx.x] += slive[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out4[0] = slive[0]; out4[1] = smin[0]; out4[2] = smax[0]; out4[3] = ssum[0]; }
}

extern "C" afqmc_status afqmc_stats(afqmc_ctx* ctx, double* out, int len) {
    if (!ctx || !out || len < 0) return fail(AFQMC_ERR_ARG, "bad arguments");
    unsigned long long c[16];
    double ws4[4];
    int status = 0;
    weight_stats_kernel<<<1, 256, 0, ctx->stream>>>(ctx->d.W, ctx->ws.weight, ctx->ws.reduce + 4); count_launches(1);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c, ctx->ws.counters, sizeof c, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ws4, ctx->ws.reduce + 4, sizeof ws4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&status, ctx->ws.status, sizeof status, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double v[14] = {(double)c[0], (double)c[1], (double)c[2], ws4[0], (double)status, ws4[1], ws4[2], ws4[3],
                    (double)c[5], (double)c[6], (double)c[7], (double)c[8], (double)c[9], (double)c[10]};
    for (int i = 0; i < len && i < 14; ++i) out[i] = v[i];
    return (status & STATUS_TIMEOUT) ? status_result(status) : AFQMC_OK;
}

extern "C" afqmc_status afqmc_energy_paths(afqmc_ctx* ctx, int rounds, int sweeps, double* e_mix, double* e_walker,
                                           double* ratio) {
    if (!ctx || !e_mix) return fail(AFQMC_ERR_ARG, "ctx and e_mix must not be NULL");
    if (rounds < 1 || sweeps < 0) return fail(AFQMC_ERR_ARG, "rounds must be >= 1 and sweeps >= 0");
    if (ctx->ws.rc) return fail(AFQMC_ERR_ARG, "measurement paths are not available with rcache = 1");
    const Dims& d = ctx->d;
    Workspace& w = ctx->ws;
    cudaStream_t s = ctx->stream;
    afqmc_status st = measure(ctx);   // at the propagation's paths
    if (st != AFQMC_OK) return st;
    CK(cudaMemcpyAsync(w.xsave, w.x, (size_t)d.pairs * d.K * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(w.Phisave, w.Phi, (size_t)d.pairs * phi_stride(d) * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(w.msum0, w.sumS, (size_t)d.W * 16, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(w.logov_cur, w.logov, (size_t)d.pairs * 16, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(w.macc, 0, (size_t)d.W * 2 * 16, s));
    CK(meas_alive(s, d, ctx->cfg.kill_threshold, w.weight, w.msum0, w.alive));
    for (int r = 0; r < rounds && st == AFQMC_OK; ++r) {
        for (int m = 0; m < sweeps && st == AFQMC_OK; ++m)   // the learned proposal gives way to the prior
            st = mcmc_sweep(ctx, w.phi, TAG_MEAS_PROPOSE, TAG_MEAS_ACCEPT, (uint32_t)(r * sweeps + m), true);
        if (st == AFQMC_OK) st = measure(ctx);
        if (st == AFQMC_OK) CK(meas_accumulate(s, d, w.logov, w.epair, w.alive, w.macc));
    }
    // the propagation's paths back; the measurement's acceptances are not the step's
    CK(cudaMemcpyAsync(w.x, w.xsave, (size_t)d.pairs * d.K * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(w.Phi, w.Phisave, (size_t)d.pairs * phi_stride(d) * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(w.counters + 3, 0, 2 * 8, s));
    ctx->measured = false;
    if (st != AFQMC_OK) return st;
    CK(meas_finish(s, d, rounds, w.weight, w.msum0, w.alive, w.macc, w.mout));
    double2 AB[2];
    CK(cudaMemcpyAsync(AB, w.mout + 2 * d.W, sizeof AB, cudaMemcpyDeviceToHost, s));
    if (e_walker) CK(cudaMemcpyAsync(e_walker, w.mout, (size_t)d.W * 16, cudaMemcpyDeviceToHost, s));
    if (ratio) CK(cudaMemcpyAsync(ratio, w.mout + d.W, (size_t)d.W * 16, cudaMemcpyDeviceToHost, s));
    int status = 0;
    if ((st = read_status(ctx, &status)) != AFQMC_OK) return st;
    const double bb = AB[1].x * AB[1].x + AB[1].y * AB[1].y;
    *e_mix = bb > 0.0 ? (AB[0].x * AB[1].x + AB[0].y * AB[1].y) / bb : 0.0;   // Re(A / B)
    return status_result(status);
}

static const uint64_t STATE_MAGIC = 0x4146514D43535431ull;

static size_t state_bytes(const Dims& d) {
    return 8 * 8 + (size_t)d.W * d.N * d.nt * 16 + (size_t)d.W * 8 + (size_t)d.pairs * d.K * 8 +
           (size_t)d.pairs * phi_stride(d) * 8;
}

extern "C" afqmc_status afqmc_state_save(afqmc_ctx* ctx, void* buf, size_t* len) {
    if (!ctx || !len) return fail(AFQMC_ERR_ARG, "bad arguments");
    const Dims& d = ctx->d;
    size_t need = state_bytes(d);
    if (!buf) { *len = need; return AFQMC_OK; }
    if (*len < need) return fail(AFQMC_ERR_STATE, "state buffer needs %zu bytes", need);
    char* p = (char*)buf;
    unsigned long long step = 0;
    CK(cudaMemcpyAsync(&step, ctx->ws.counters, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    uint64_t hdr[8] = {STATE_MAGIC, (uint64_t)d.N, (uint64_t)d.nu, (uint64_t)d.nd, (uint64_t)d.K, (uint64_t)d.W,
                       (uint64_t)d.P, step};
    memcpy(p, hdr, sizeof hdr);
    p += sizeof hdr;
    size_t b;
    CK(cudaMemcpyAsync(p, ctx->ws.phi, b = (size_t)d.W * d.N * d.nt * 16, cudaMemcpyDeviceToHost, ctx->stream)); p += b;
    CK(cudaMemcpyAsync(p, ctx->ws.weight, b = (size_t)d.W * 8, cudaMemcpyDeviceToHost, ctx->stream)); p += b;
    CK(cudaMemcpyAsync(p, ctx->ws.x, b = (size_t)d.pairs * d.K * 8, cudaMemcpyDeviceToHost, ctx->stream)); p += b;
    CK(cudaMemcpyAsync(p, ctx->ws.Phi, b = (size_t)d.pairs * phi_stride(d) * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *len = need;
    return AFQMC_OK;
}

extern "C" afqmc_status afqmc_state_load(afqmc_ctx* ctx, const void* buf, size_t len) {
    if (!ctx || !buf) return fail(AFQMC_ERR_ARG, "bad arguments");
    const Dims& d = ctx->d;
    if (len != state_bytes(d)) return fail(AFQMC_ERR_STATE, "state has %zu bytes, expected %zu", len, state_bytes(d));
    uint64_t hdr[8];
    memcpy(hdr, buf, sizeof hdr);
    if (hdr[0] != STATE_MAGIC || hdr[1] != (uint64_t)d.N || hdr[2] != (uint64_t)d.nu || hdr[3] != (uint64_t)d.nd ||
        hdr[4] != (uint64_t)d.K || hdr[5] != (uint64_t)d.W || hdr[6] != (uint64_t)d.P)
        return fail(AFQMC_ERR_STATE, "state header does not match this context");
    const char* p = (const char*)buf + sizeof hdr;
    size_t b;
    CK(cudaMemcpyAsync(ctx->ws.phi, p, b = (size_t)d.W * d.N * d.nt * 16, cudaMemcpyHostToDevice, ctx->stream)); p += b;
    CK(cudaMemcpyAsync(ctx->ws.weight, p, b = (size_t)d.W * 8, cudaMemcpyHostToDevice, ctx->stream)); p += b;
    CK(cudaMemcpyAsync(ctx->ws.x, p, b = (size_t)d.pairs * d.K * 8, cudaMemcpyHostToDevice, ctx->stream)); p += b;
    CK(cudaMemcpyAsync(ctx->ws.Phi, p, b = (size_t)d.pairs * phi_stride(d) * 8, cudaMemcpyHostToDevice, ctx->stream));
    unsigned long long c[16] = {hdr[7]};
    CK(cudaMemcpyAsync(ctx->ws.counters, c, sizeof c, cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->ws.rdirty) CK(set_int(ctx->stream, ctx->ws.rdirty, d.pairs, 1));   // every cached matrix is stale
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->steps_taken = (long long)hdr[7];
    ctx->measured = false;
    return AFQMC_OK;
}

extern "C" void afqmc_destroy(afqmc_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    if (ctx->prof_events) {
        for (int i = 0; i < ctx->prof_cap; ++i) cudaEventDestroy(ctx->prof_events[i]);
        free(ctx->prof_events);
        free(ctx->prof_phase);
    }
    free(ctx);
    cudaGetLastError();   // nothing to report from here: leave no error pending for the next call
}

__global__ void philox_fill_kernel(uint32_t* out, int64_t n, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                   uint32_t k0, uint32_t k1) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Philox4 r = philox4x32_10(c0 + (uint32_t)i, c1, c2, c3, k0, k1);
    out[4 * i + 0] = r.w[0];
    out[4 * i + 1] = r.w[1];
    out[4 * i + 2] = r.w[2];
    out[4 * i + 3] = r.w[3];
}

extern "C" afqmc_status afqmc_philox_fill(uint32_t* out, int64_t n, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          uint64_t key, void* stream) {
    if (!out || n < 0) return fail(AFQMC_ERR_ARG, "bad arguments");
    if (n == 0) return AFQMC_OK;
    philox_fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(out, n, c0, c1, c2, c3,
                                                                                     (uint32_t)key, (uint32_t)(key >> 32)); count_launches(1);
    CK(cudaGetLastError());
    return AFQMC_OK;
}
