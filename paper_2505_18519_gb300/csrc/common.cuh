// Shared device helpers of the AFQMC library: complex arithmetic on double2,
// the counter-based generator, and the context/workspace layout.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/afqmc.h"

namespace afq {

// ---------------------------------------------------------------- complex helpers
__host__ __device__ __forceinline__ double2 cmk(double re, double im) { return make_double2(re, im); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return cmk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return cmk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return cmk(a.x, -a.y); }
// a += b * c
__host__ __device__ __forceinline__ void cfma(double2& a, double2 b, double2 c) {
    a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
    a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}
__device__ __forceinline__ double cabs_(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    // Smith's algorithm
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return cmk((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.x * r + b.y;
        return cmk((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__device__ __forceinline__ double2 cexp_(double2 z) {
    double s, c;
    sincos(z.y, &s, &c);
    double m = exp(z.x);
    return cmk(m * c, m * s);
}

// ---------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11): ten rounds,
// each multiplying counter words 0 and 2 by fixed odd constants and mixing
// the products' halves with words 1, 3 and the round key; the key advances by
// two Weyl increments between rounds.
struct Philox4 { uint32_t w[4]; };

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                         uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint32_t lo0 = M0 * c0, hi0 = mulhi32(M0, c0);
        uint32_t lo1 = M1 * c2, hi1 = mulhi32(M1, c2);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    Philox4 o; o.w[0] = c0; o.w[1] = c1; o.w[2] = c2; o.w[3] = c3;
    return o;
}

// Random-stream tags (counter word 3 = tag << 24 | sweep).
enum : uint32_t {
    TAG_INIT_WALKER = 1, TAG_INIT_PATH = 2, TAG_FIELD = 3, TAG_PROPOSE = 4,
    TAG_ACCEPT = 5, TAG_BURN_PROPOSE = 6, TAG_BURN_ACCEPT = 7, TAG_MLP_INIT = 9, TAG_COMB = 10,
    TAG_MEAS_PROPOSE = 11, TAG_MEAS_ACCEPT = 12
};

__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
    uint64_t v = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
    return (double)v * 0x1.0p-53;
}

// Block j of a draw: counter = (j, entity, step, tag<<24|sweep).
__device__ __forceinline__ Philox4 stream_block(uint64_t seed, uint32_t tag, uint32_t step, uint32_t entity,
                                                uint32_t sweep, uint32_t j) {
    return philox4x32_10(j, entity, step, (tag << 24) | (sweep & 0xFFFFFFu), (uint32_t)seed,
                         (uint32_t)(seed >> 32));
}

// Two standard normals (Box-Muller) from block j: numbers 2j and 2j+1 of the draw.
__device__ __forceinline__ double2 normal_pair(uint64_t seed, uint32_t tag, uint32_t step, uint32_t entity,
                                              uint32_t sweep, uint32_t j) {
    Philox4 b = stream_block(seed, tag, step, entity, sweep, j);
    double u0 = u53(b.w[0], b.w[1]), u1 = u53(b.w[2], b.w[3]);
    double r = sqrt(-2.0 * log1p(-u0));
    double s, c;
    sincospi(2.0 * u1, &s, &c);
    return cmk(r * c, r * s);
}

__device__ __forceinline__ double normal_at(uint64_t seed, uint32_t tag, uint32_t step, uint32_t entity,
                                           uint32_t sweep, uint32_t idx) {
    double2 z = normal_pair(seed, tag, step, entity, sweep, idx >> 1);
    return (idx & 1) ? z.y : z.x;
}

__device__ __forceinline__ double uniform_at0(uint64_t seed, uint32_t tag, uint32_t step, uint32_t entity,
                                             uint32_t sweep) {
    Philox4 b = stream_block(seed, tag, step, entity, sweep, 0);
    return u53(b.w[0], b.w[1]);
}

// ---------------------------------------------------------------- status word bits
enum : int { STATUS_SINGULAR = 1, STATUS_NONFINITE = 2, STATUS_TIMEOUT = 4 };

// ---------------------------------------------------------------- learned proposal buffers
struct MlpBuffers {
    int Kp, Wp;                        // K and W rounded up to 16
    double* UPhi0;                     // K x N x n_up, U_k Phi0
    double2* Theta0;                   // W x N x nt, phi (Phi0^T phi)^-1
    double2* logdet0;                  // W x 2
    float* featf;                      // Wp x Kp
    __nv_bfloat16* featb;              // Wp x Kp
    float *theta, *adam_m, *adam_v, *grad;   // flat parameters, moments, gradient
    __nv_bfloat16 *W1b, *W2b, *W3b;    // H x Kp, H x H, 2Kp x H
    float *Zf, *H1f, *H2f, *dHf, *dZf; // Wp x H
    __nv_bfloat16 *H1b, *H2b, *dZb;    // Wp x H
    float *outf, *doutf;               // Wp x 2Kp
    __nv_bfloat16* doutb;              // Wp x 2Kp
    float *mu, *logv, *logv_raw;       // W x K
    float *gW1p, *gb1, *gW2, *gb2, *gW3p, *gb3p;   // padded weight gradients, bias sums
    double *loss_part, *loss;          // W, 1
    unsigned long long* counter;       // Adam steps taken
    int* status;                       // the context's device status word (a GEMM's wait that gave up)
};

// ---------------------------------------------------------------- workspace layout
// Every buffer of a context lives in the caller's workspace, 256-byte aligned.
struct Workspace {
    // Hamiltonian and trial (copied at init)
    double* h;        // N*N
    double* L;        // G*N*N
    double* Phi0;     // N*n_up
    double* U;        // KU*N*N (the operators U_k of one slice)
    double* Pslice;   // N*N propagator between slices of a multi-slice trial (or null)
    double2* Vtmp;    // pairs*N*n_up complex work of the multi-slice chain (or null)
    void* Udf;        // K*N*N double-float copy of U (mixed-precision path)
    double* T;        // N*N, h - 1/2 sum_g L_g L_g
    double* expT;     // N*N, exp(-tau T / 2)
    void* Ldf;        // G*N*N double-float copy of L (mixed-precision path)
    void* hdf;        // N*N double-float copy of h (refinement of the mixed path)
    void* xdf;        // max(W*P*K, 2W*G) double-float coefficients of the double-float GEMMs (mixed path)
    void* expTdf;     // N*N double-float copy of expT (mixed-precision path)
    double* scratchNN;  // 3*N*N for the matrix exponential at init
    void* Lt;           // split-BF16 image of (h, L_g) for the tensor-core contraction
    void* Yimg;         // split images of Y_g = X_g phi_w per walker (walker-side tensor-core form)
    void* tcw;          // work of the general walker-side tensor-core form (contract_tcw.cu)
    void* ywalk;        // Y_g = X_g phi_w of every walker, and the walkers' orbitals as columns (walker-side FP64 form)
    // composite walkers
    double2* phi;     // W*N*nt (nt = n_up + n_dn)
    double* weight;   // W
    double* x;        // W*P*K
    double* Phi;      // W*P*N*n_up
    // per step, per pair
    double2* logdet;     // W*P*2   per spin, at phi
    double2* logov;      // W*P     sum over spins, at phi
    double2* Theta;      // W*P*N*nt
    double2* vpair;      // W*P*G
    double2* epair;      // W*P
    double2* logdet_new; // W*P*2   at phi'
    double2* logov_cur;  // W*P     current paths at phi'
    // per step, per walker
    double2* sumS;    // W
    double2* vbar;    // W*G
    double2* ebar;    // W
    double2* y;       // W*G   x - xbar
    double2* logshift;  // W  sum_g (xi xbar - xbar^2/2)
    // error-controlled FP64 refinement of the tensor-core contraction (null when off)
    double* refine_th2;   // W*P   ||Theta_p||_F^2
    int* refine_items;    // W*P   pairs to recompute in FP64
    int* refine_n;        // 1     their number
    double* refine_lam;   // G+1   ||L_g||_2^2, then their sum at [G]
    int* cheb_redo;       // W*P+1 trial orbitals to redo in double-float (tensor-core kernel), count at [W*P]
    // double-float copies for the overlaps' products on the mixed path (null when not used):
    void* Phidf;          // W*P*N*n_up  8-byte pairs: Phi at a measurement, then Phi(x') in a sweep
    void* phidf;          // W*N*nt      16 bytes per complex entry: the walkers the overlap reads
    void* Aov;            // W*P*(n_up^2+n_dn^2) 16-byte double-float entries: A_p from the tensor cores
    void* Uimg;           // digit images of U and its column exponents (proposal matrices on the tensor cores)
    double* Aplanes;  // 2W*N*N  rows 2w: sum_g Re(y) L_g ; 2w+1: sum_g Im(y) L_g
                      //         (double-float pairs, 8 bytes each, on the mixed-precision path)
    double2* phi_new; // W*N*nt
    double2* propbuf; // W*2*N*nt work space of the propagation when it does not fit in shared memory (else null)
    double2* old_sum; // W   sum_p S_p ov'/ov
    double2* ratio;   // W
    double* Iabs;     // W
    int* alive;       // W
    // population control (null when off)
    double* comb_cum; // W   running sums of the weights
    int* comb_hit;    // W   whether a tooth picked the walker
    int* comb_slot;   // W   walker of every tooth, then the replaced slots
    int* comb_from;   // W   walker each replaced slot copies
    int* comb_flag;   // 2   whether this step combed, replaced walkers
    // extra measurement paths: the propagation's paths while the measurement's move
    double* xsave;    // W*P*K
    double* Phisave;  // W*P*N*n_up
    double2* msum0;   // W    sum_p S_p of the propagation's paths
    double2* macc;    // 2W   sum S' E_L, sum S' over the measurement paths
    double2* mout;    // 2W+2 E'_w, R_w, sum W R E', sum W R
    // cached half-rotated matrices X_g Phi_p (FP64 path, null when off)
    double* rc;       // W*P*(G+1)*N*n_up
    int* rdirty;      // W*P  1: the pair's path moved since its matrices were formed
    int* rlist;       // W*P  pairs to refresh
    int* rcount;      // 1
    // Metropolis
    double* xprop;    // W*P*K
    double* Sprop;    // W*P*N*N   sum_k x'_k U_k
    double* Phiprop;  // W*P*N*n_up
    double2* logdet_prop; // W*P*2
    // accounting
    double* history;  // capacity*4
    double* reduce;   // 8 doubles of scratch for reductions
    unsigned long long* counters;  // 16: [0] step, [1] accepted (total), [2] proposed (total), [3] accepted this step
    int* status;      // 1 int
    MlpBuffers mlp;   // learned proposal (only with AFQMC_PROPOSAL_MLP)
    size_t total;
};

struct Dims {
    int N, nu, nd, nt, G, K, W, P;
    long long pairs;
    // launch shapes chosen by the autotuner (0 = built-in default)
    int ov_wpb;        // warps (matrices) per block of the overlap kernel
    int tc_tp;         // pairs per block of the tensor-core contraction
    int cheb_threads;  // threads per block of the trial-orbital kernel
    // polls of an mbarrier before a tensor-core kernel's main wait gives up (sets
    // STATUS_TIMEOUT, drains its copies and MMAs with their own fixed bound, returns)
    uint32_t wait_polls = 1u << 26;
    // complex trial orbitals (the complex or multi-slice trial, FP64 path): Phi is
    // stored as N x n_up complex values per pair; K then counts the hidden
    // variables of one sample (slices x the operators' count KU)
    int cphi = 0;
    int KU = 0;        // operators U_k (0: K)
    int slices = 1;
};

// Doubles per pair of the trial orbitals Phi (N x n_up, real or complex).
inline long long phi_stride(const Dims& d) { return (long long)d.N * d.nu * (d.cphi ? 2 : 1); }

}  // namespace afq

namespace afq {
// Process-wide count of kernel launches made by this library.
void count_launches(long long n);
// Raises the dynamic shared-memory limit of `kernel` on the current device to at
// least `bytes`.  A block may use 48 KB of shared memory in all (static plus
// dynamic) without this opt-in, so every launch with dynamic shared memory goes
// through here.  The limit only ever grows, so kernels captured earlier into a
// graph with a larger size stay launchable.
cudaError_t raise_smem_limit(const void* kernel, size_t bytes);
// Phases of a step timed by afqmc_profile (CUDA events on the context's stream).
enum Phase : int {
    PH_OVERLAP = 0, PH_CONTRACT, PH_AVERAGE, PH_FIELDS, PH_PROPAGATE, PH_RATIO, PH_PROPOSE, PH_TRIAL,
    PH_MCMC_OVERLAP, PH_ACCEPT, PH_FINISH, PH_COMB, PH_REFINE, PH_COUNT
};
}  // namespace afq

struct afqmc_ctx {
    afqmc_config cfg;
    afq::Dims d;
    afq::Workspace ws;
    cudaStream_t stream;
    long long steps_taken;   // host mirror of the device step counter
    bool measured;           // afqmc_energy has filled the per-pair buffers
    // profiling: events recorded at phase boundaries while enabled
    bool profiling;
    int prof_used, prof_cap;
    cudaEvent_t* prof_events;   // prof_cap events
    int* prof_phase;            // phase that ends at event i (-1: a step start)
    double prof_ms[afq::PH_COUNT];
    long long prof_launches[afq::PH_COUNT];
    long long prof_steps;
};
