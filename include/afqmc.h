/*
 * afqmc.h -- C ABI of the GB300 library for phaseless auxiliary-field quantum
 * Monte Carlo with a stochastically sampled (hidden-variable) trial wave
 * function (arXiv 2505.18519).
 *
 * The paper's method (Sec. III A, Appendix B.2): every random walker phi_w is
 * tethered to P Metropolis paths x_wp over the trial's hidden variables; the
 * trial sample of a path is the Slater determinant
 *     Phi(x) = exp(sum_k x_k U_k) Phi0                      (Eq. (20)-(21), one slice)
 * and one leapfrog step
 *   (1) measures, for every pair (w, p), the overlap det(Phi^T phi), the mixed
 *       Green's function, the force-bias values <L_g> and the local energy,
 *       and averages them over the paths with the path signs S_p (Eq. (25)-(27));
 *   (2) propagates phi_w by B(x - xbar) (Eq. (5), (12), (15)) and updates the
 *       weight with the phaseless importance function (Eq. (14), (17));
 *   (3) re-equilibrates the paths by Metropolis against the new walker
 *       (Eq. (23)) and applies the hand-off constraint (Eq. (28)-(29));
 *   (4) re-orthonormalises the walkers.
 *
 * Conventions for every entry point
 *   - Arrays are row-major, FP64 (complex numbers as interleaved re, im pairs).
 *   - "Host or device pointer": any pointer the CUDA runtime can copy from with
 *     cudaMemcpyDefault (pageable or pinned host memory, or device memory).
 *   - The caller owns every array it passes; the library copies what it needs
 *     before the call returns and never keeps a caller pointer, except the
 *     device workspace given to afqmc_init, which must stay allocated until
 *     afqmc_destroy.
 *   - The library never calls cudaMalloc/cudaFree: all device memory it uses
 *     is the caller's workspace.  Host memory for the context is malloc'ed.
 *   - Every call returns a status and never aborts the process.  Device-side
 *     numerical problems (a singular overlap, a non-finite weight) set a
 *     device status word that afqmc_energy and afqmc_stats report.
 *   - Work is enqueued on the CUDA stream given at init; calls that return
 *     values to the host synchronise that stream.
 *   - Not thread-safe per context; distinct contexts are independent.
 */
#ifndef AFQMC_H
#define AFQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afqmc_ctx afqmc_ctx;

typedef enum {
    AFQMC_OK = 0,
    AFQMC_ERR_ARG = 1,        /* invalid argument, or a size the library does not support */
    AFQMC_ERR_CUDA = 2,       /* a CUDA runtime call failed (the message says which) */
    AFQMC_ERR_WORKSPACE = 3,  /* workspace missing, too small, or not 256-byte aligned */
    AFQMC_ERR_NUMERIC = 4,    /* the device flagged a singular overlap or a non-finite value */
    AFQMC_ERR_STATE = 5,      /* a state buffer of the wrong size or shape */
    AFQMC_ERR_TIMEOUT = 6     /* a tensor-core kernel gave up a bounded wait (see wait_polls); its
                                 results of that measurement are not valid, the context stays usable */
} afqmc_status;

/* weight update of the hand-off (Sec. III A, Eq. (17), (29)) */
enum {
    AFQMC_CONSTRAINT_COMBINED = 0,   /* W *= |I| max(0, cos(dtheta + dtheta_T)) (default) */
    AFQMC_CONSTRAINT_SEPARATE = 1,   /* W *= |I| max(0, cos dtheta) max(0, cos dtheta_T) */
    AFQMC_CONSTRAINT_HALF_PLANE = 2  /* W *= |I| max(0, cos dtheta), and W = 0 if |dtheta_T| > pi/2 */
};

/* importance function |I| of the weight update (Sec. III A); the phase dtheta of
 * the constraint comes from the overlap ratio Eq. (25) in both */
enum {
    AFQMC_IMPORTANCE_HYBRID = 0,       /* |I| of Eq. (14): |p(x - xbar)/p(x)| times the ratio Eq. (25) (default) */
    AFQMC_IMPORTANCE_LOCAL_ENERGY = 1  /* |I| = exp(-tau Re E_w), E_w of Eq. (27) at the start of the step */
};

/* Metropolis proposal for the paths (Sec. III A; Appendix B.2) */
enum {
    AFQMC_PROPOSAL_PRIOR = 0,  /* independent draw x' ~ N(0, I) (the paper's sampler) */
    AFQMC_PROPOSAL_PCN = 1,    /* x' = sqrt(1 - beta^2) x + beta xi, xi ~ N(0, I) */
    AFQMC_PROPOSAL_RW = 2,     /* Gaussian random walk x' = x + rw_step xi */
    AFQMC_PROPOSAL_MLP = 3     /* learned proposal N(mu(f_w), diag v(f_w)) of an MLP on walker features,
                                  mixed with the random walk (probability mlp_mix); burn-in uses the prior */
};

/* arithmetic of the two big contractions (R = Phi^T L_g and M = R Theta) */
enum {
    AFQMC_PRECISION_FP64 = 0,  /* FP64 everywhere.  N <= 256, n_up <= 64, n_up^2 + n_dn^2 <= 4096, and
                                  3 N n_up <= 25600 (e.g. N = 200 with 40 + 40 electrons) */
    AFQMC_PRECISION_BF16X3 = 1, /* the fused contraction on the tensor cores in split BF16 (hi*hi + hi*lo +
                                   lo*hi, FP32 accumulation, traces summed in FP64); trial orbitals, proposal
                                   and field matrices and the propagation in double-float (pairs of FP32
                                   numbers, about 44 bits; the propagation in FP64 when its 2 N (n_up + n_dn)
                                   complex work values exceed shared memory); everything else FP64.
                                   N <= 128, n_up <= 32 */
    AFQMC_PRECISION_FP16X3 = 2, /* the same with each operand row/column scaled by a power of two and split
                                   into an integer FP16 part (|x| <= 256) and an FP16 remainder (about 20 bits
                                   relative to the row's largest entry); integer*integer products go to their
                                   own, exact accumulator, the three correction products to a second one */
    AFQMC_PRECISION_FP16X6 = 3  /* the walker-side tensor-core form (tc_form AUTO or WALKER) only: each operand
                                   split into the integer FP16 part and two FP16 remainders (about 31 bits),
                                   six products per real product (every one above about 2^-28 of the
                                   integer*integer term), the entries reaching the traces as FP32 numbers (about
                                   24 bits).  The GEMM-Y block keeps three parts of the walker's orbitals
                                   (2 n_up rows rounded up to 8, per K chunk of 64) in shared memory, and
                                   the GEMM-Z block three parts of a walker tile: N <= 256 with
                                   n_up <= 40 */
};

typedef struct {
    int N;              /* orbitals (basis size) */
    int n_up, n_dn;     /* electrons per spin; 0 <= n_dn <= n_up, n_up >= 1 */
    int n_chol;         /* Cholesky vectors Gamma (Eq. (3)) */
    int K;              /* hidden variables of the trial */
    int n_walkers;      /* W */
    int n_paths;        /* P, paths tethered to each walker */
    int n_sweeps;       /* Metropolis sweeps M per step (>= 1) */
    int n_burn;         /* Metropolis sweeps at fixed walkers during afqmc_init (>= 0) */
    int constraint;     /* AFQMC_CONSTRAINT_* */
    int proposal;       /* AFQMC_PROPOSAL_* */
    int precision;      /* AFQMC_PRECISION_* */
    int taylor_order;   /* order of the auxiliary-field propagator's Taylor series (6) */
    int history_capacity; /* per-step energy records kept on the device (ring buffer, >= 1) */
    double dtau;        /* imaginary time step tau > 0 */
    double pcn_beta;    /* beta of the pCN proposal, 0 < beta <= 1 */
    double e_shift;     /* constant E_T: every step multiplies weights by exp(tau E_T) */
    double kill_threshold; /* a walker whose |sum_p S_p| is below this gets weight 0 */
    uint64_t seed;      /* key of the Philox4x32-10 streams */
    int64_t walker_offset; /* global index of walker 0 in the random streams: walker w draws as
                              walker walker_offset + w, so shards of one population on several
                              GPUs reproduce the single-GPU run exactly */
    double rw_step;     /* random-walk step (AFQMC_PROPOSAL_RW, and the fallback of AFQMC_PROPOSAL_MLP) */
    double mlp_mix;     /* probability of a random-walk move under AFQMC_PROPOSAL_MLP */
    double mlp_lr;      /* Adam learning rate of the proposal network */
    int mlp_train;      /* 1: after every step, one Adam step on the paths' states (online training) */
    double refine_tol;  /* mixed precision, per-pair tensor-core form: per-walker energy tolerance (Ha) of
                           the error-controlled refinement.  Each measurement estimates every pair's
                           contraction error as (2/N) u sum_g ||L_g||_2^2 ||Theta_p||_F^2 (u = 2^-20; fp16x6:
                           2^-24) and recomputes
                           in double-float (FP32 pairs, about 44 bits) the pairs with the largest ||Theta_p||_F
                           until the estimated error of the
                           walker's average, 2 sqrt(sum of the kept pairs' squared errors) / |sum_p S_p|,
                           is at most refine_tol / 2.  0 turns it off.  Default 1e-4.  Not used by the
                           walker-side tensor-core form (N <= 64, n_up + n_dn <= 40), which keeps no Theta */
    int importance;     /* AFQMC_IMPORTANCE_* (default hybrid) */
    int pop_period;     /* population control of the branching random walk (Sec. II B, II D): after every
                           pop_period-th step a comb resamples the W walkers (phi, paths x and Phi(x)) in
                           proportion to their weights and gives each the mean weight; teeth spaced sum W / W
                           apart from u sum W / W, u a Philox uniform (tag 10, entity walker_offset, the
                           step's index).  0 (default) turns it off; on, n_walkers <= 65535.  Each GPU of a
                           sharded run combs its own walkers */
    int rcache;         /* 1: precision FP64 with the half-rotated matrices X_g Phi(x_wp) (g = h, L_1 ..)
                           cached per pair and refreshed only for the paths whose Metropolis move was accepted
                           since the last measurement; the contraction is then M = R Theta (2 N (n_up^2 +
                           n_dn^2) multiply-adds per pair and matrix).  Costs (n_chol + 1) N n_up doubles of
                           workspace per pair (16.4 GB for 512 x 32 pairs of the 50-orbital system) and needs
                           4 warps' shares of Theta (N x (n_up + n_dn) complex) and one matrix (N x n_up) in
                           220 KB of shared memory, and the refresh N^2 + 8 N n_up doubles in 200 KB (with
                           10 + 10 electrons N <= 124; not 120 orbitals with 24 + 24).  0 (default): off */
    int64_t wait_polls; /* tensor-core kernels: polls of an mbarrier before a main wait (a copy landing,
                           MMAs completing, an epilogue freeing a buffer) gives up; the block then sets
                           bit 4 of the device status word, lets its own copies and MMAs complete (a
                           fixed bound of 2^22 polls each) and returns, and afqmc_energy / afqmc_stats
                           return AFQMC_ERR_TIMEOUT.  0 (default): 2^26 polls; at most 2^31 */
    int tc_form;        /* mixed precision: which tensor-core form runs the contraction.
                           AFQMC_TC_AUTO (0, default): the walker-side form of N <= 64 with
                           n_up + n_dn <= 40, else the per-pair form (N <= 128, n_up <= 32; it has the
                           error-controlled refinement), else the general walker-side form;
                           AFQMC_TC_PER_PAIR (1); AFQMC_TC_WALKER (2): the general walker-side form
                           (N <= 256, n_up <= 64; refined like the per-pair form).  Precision FP16X6
                           always takes the general walker-side form */
    double trial_alpha_re, trial_alpha_im;   /* alpha of the trial samples (default 1 + 0i) */
    int trial_slices;   /* hidden-variable slices of a trial sample (default 1).  The samples are
                           Phi(x) = exp(alpha S_m) P ... P exp(alpha S_1) Phi0 with S_l = sum_k x_lk U_k
                           and K hidden variables per slice (x has trial_slices K entries): the
                           complex VAFQMC form of Eq. (30) (alpha = -i sqrt(s), U_k = L_k) and the
                           multi-slice form of Eq. (19), (32) (P from afqmc_init_trial).  Any value other
                           than alpha = 1, one slice needs precision FP64, a proposal other than the
                           learned one, rcache = 0, and 48 N n_up bytes of shared memory at most
                           200 KB; Phi is then stored and returned as complex (state buffer) */
    int trial_form;     /* mixed precision: how the trial orbitals exp(S) Phi0 of Eq. (20)-(21) are formed.
                           AFQMC_TRIAL_TC (2): the Chebyshev products S V on the tensor cores (each operand
                           split into five 8-bit integer digits, the digit products of orders 0-5
                           accumulated exactly in FP32, combined in double-float: about 40 bits), one
                           proposal per SM, where N <= 128 and n_up <= 32, else as AFQMC_TRIAL_DF;
                           AFQMC_TRIAL_DF (1): the whole recurrence in double-float arithmetic (about 44
                           bits) on the CUDA cores, several proposals per SM; AFQMC_TRIAL_AUTO (0,
                           default): the tensor cores for 64 < N <= 128, else double-float (measured: the
                           tensor-core form is 5.9x faster at N = 120, 2.2x slower at N = 50) */
    int overlap_form;   /* mixed precision, real trial: how the overlap matrices A_p = Phi_p^T phi_w behind
                           the path signs and ratios (Eq. (25)-(26)) are formed.  AFQMC_OVERLAP_AUTO (0,
                           default): on the tensor cores (each operand split into five 8-bit integer
                           digits, the digit products of orders 0-4 accumulated exactly in FP32, combined
                           in double-float: about 40 bits) where N <= 128 and n_up <= 40, else as
                           AFQMC_OVERLAP_DF; AFQMC_OVERLAP_DF (1): compensated double-float sums on the
                           CUDA cores (about 44 bits).  The LU, log-determinants and inverses are FP64
                           either way */
} afqmc_config;

enum { AFQMC_TRIAL_AUTO = 0, AFQMC_TRIAL_DF = 1, AFQMC_TRIAL_TC = 2 };
enum { AFQMC_OVERLAP_AUTO = 0, AFQMC_OVERLAP_DF = 1 };

enum { AFQMC_TC_AUTO = 0, AFQMC_TC_PER_PAIR = 1, AFQMC_TC_WALKER = 2 };

/* Fill *cfg with defaults (combined constraint, prior proposal, FP64, Taylor
 * order 6, one sweep, 20 burn-in sweeps, kill threshold 1e-10, refine_tol 1e-4)
 * and zero sizes. */
void afqmc_config_default(afqmc_config* cfg);

/* Bytes of device workspace the configuration needs (0 if cfg is invalid).  Besides
 * the state and per-pair buffers it holds, for the walker-side contraction forms,
 * Y_g = L_g phi_w of every walker: (n_chol + 1) N 2 (n_up + n_dn) doubles per walker
 * in FP64 (4 MB per walker on the 50-orbital system), or the split-FP16 images
 * of it (6.2 MB per walker there). */
size_t afqmc_workspace_bytes(const afqmc_config* cfg);

/* Create a context.
 *   h     N*N          one-body matrix h_ij (symmetric)                 host or device
 *   L     n_chol*N*N   Cholesky vectors L_g,ij (each symmetric), so that
 *                      V_ijkl = sum_g L_g,ij L_g,kl (Eq. (1), (3))        host or device
 *   Phi0  N*n_up       trial orbitals (spin down uses the first n_dn)    host or device
 *   U     K*N*N        hidden-variable operators U_k (each symmetric)    host or device
 *   workspace, workspace_bytes: device memory of at least
 *                      afqmc_workspace_bytes(cfg) bytes, 256-byte aligned,
 *                      owned by the caller, kept alive until afqmc_destroy
 *   stream             cudaStream_t to run on (NULL = legacy default stream)
 * It forms T = h - 1/2 sum_g L_g L_g and exp(-tau T/2), draws the initial
 * walkers phi_w = orthonormalised Phi(x_w) and paths x_wp from the prior, sets
 * W = 1, runs n_burn Metropolis sweeps, and synchronises the stream.
 * The step counter starts at 0.  On error *out is NULL. */
afqmc_status afqmc_init(const afqmc_config* cfg, const double* h, const double* L,
                        const double* Phi0, const double* U, void* workspace,
                        size_t workspace_bytes, void* stream, afqmc_ctx** out);

/* afqmc_init for a multi-slice trial (trial_slices > 1): slice_prop (N*N, host or
 * device, real) is the fixed propagator P between slices, e.g. exp(-t T) of the
 * ansatz of Eq. (32); NULL is allowed only with one slice. */
afqmc_status afqmc_init_trial(const afqmc_config* cfg, const double* h, const double* L, const double* Phi0,
                              const double* U, const double* slice_prop, void* workspace, size_t workspace_bytes,
                              void* stream, afqmc_ctx** out);

/* Enqueue n_steps leapfrog steps (asynchronous).  Each step first measures the
 * walkers it starts from and appends {sum_w W_w Re E_w, sum_w W_w,
 * sum_w W_w |sum_p S_p|/P, accepted moves} to the device history. */
afqmc_status afqmc_step(afqmc_ctx* ctx, int n_steps);

/* Measure the current state (no step is taken) and synchronise:
 *   e_mix     = sum_w W_w Re E_w / sum_w W_w           (Eq. (16), real part)
 *   sum_w     = sum_w W_w
 *   mean_sign = sum_w W_w |sum_p S_p| / (P sum_w W_w)  (Sec. III A, path-sign average)
 *   e_walker  (nullable) 2*W doubles: E_w = sum_p S_p E_L,wp / sum_p S_p as re, im
 * Walkers of weight 0 do not enter the sums.  Returns AFQMC_ERR_NUMERIC if the
 * device status word is set (the values are still written). */
afqmc_status afqmc_energy(afqmc_ctx* ctx, double* e_mix, double* sum_w, double* mean_sign,
                          double* e_walker);

/* Mixed energy from extra, measurement-only paths (Sec. III A, last paragraph;
 * Appendix B.3).  From the current paths, `rounds` times `sweeps` Metropolis
 * sweeps at the current walkers (Philox tags 11 and 12 with the current step's
 * index, the sweep numbered r sweeps + m; the learned proposal gives way to the
 * prior); the paths after every round count as P more samples, P' = rounds P.
 * For every walker with W > 0 and |sum_p S_p| above the kill threshold:
 *   E'_w = sum_p' S'_p' E_L,p' / sum_p' S'_p',
 *   R_w  = (sum_p' S'_p' / P') / (sum_p S_p / P),
 *   e_mix = Re( sum_w W_w R_w E'_w / sum_w W_w R_w ).
 * e_walker and ratio (nullable) receive E'_w and R_w, 2*W doubles each (re, im;
 * zero for walkers that do not count).  The propagation's paths, weights and
 * statistics are left as they were.  Synchronises.  rounds >= 1, sweeps >= 0
 * (one round without sweeps is afqmc_energy's estimate); not available with
 * rcache = 1 (AFQMC_ERR_ARG).  Returns AFQMC_ERR_NUMERIC if the device status
 * word is set. */
afqmc_status afqmc_energy_paths(afqmc_ctx* ctx, int rounds, int sweeps, double* e_mix, double* e_walker,
                                double* ratio);

/* Trial samples Phi(x) (Eq. (20)-(21): exp(sum_k x_k U_k) Phi0; the complex or
 * multi-slice forms of Eq. (19), (30) when the context has them) for n rows of
 * hidden variables, in the arithmetic the context's precision uses for its own
 * paths (FP64; mixed precision: trial_form).  Uses the proposal buffers only:
 * the walkers and paths are left as they are.
 *   x    n*K doubles, row-major, host or device
 *   out  n*N*n_up doubles (real trial) or n*N*n_up complex values (interleaved),
 *        row-major per sample, host or device
 * 0 <= n <= n_walkers * n_paths, else AFQMC_ERR_ARG.  Synchronises the stream. */
afqmc_status afqmc_trial_orbitals(afqmc_ctx* ctx, const double* x, int64_t n, double* out);

/* After afqmc_energy: copy per-pair and per-walker measurements to host arrays
 * (each nullable):
 *   logov       2*W*P       log <Phi(x_wp)|phi_w> = log|det| + i Arg det (both spins)
 *   e_local     2*W*P       local energy E_L,wp (re, im)
 *   force_bias  2*W*n_chol  path-averaged <L_g>_w (re, im), Eq. (27) */
afqmc_status afqmc_observables(afqmc_ctx* ctx, double* logov, double* e_local, double* force_bias);

/* Copy the last min(n, steps taken, capacity) per-step records, oldest first,
 * into out[4*i + {0,1,2,3}] = {sum W Re E, sum W, sum W |sum S|/P, accepted};
 * *n_out receives the count.  Synchronises. */
afqmc_status afqmc_history(afqmc_ctx* ctx, double* out, int n, int* n_out);

/* Statistics since init (synchronises); out[0..len) receives, as available:
 *   0 steps taken, 1 accepted moves, 2 proposed moves, 3 live walkers,
 *   4 device status word (0 = fine), 5 min weight, 6 max weight, 7 sum weight,
 *   8 pairs recomputed by the refinement (see refine_tol) since init,
 *   9 population-control combs applied since init (see pop_period),
 *   10 walkers those combs replaced by copies of others,
 *   11 pairs whose cached half-rotated matrices were formed since init (see rcache),
 *   12 Chebyshev terms summed by the tensor-core trial-orbital kernel since init (see
 *      trial_form), 13 trial samples it handed to the double-float kernel because
 *      the Lanczos interval missed part of the spectrum */
afqmc_status afqmc_stats(afqmc_ctx* ctx, double* out, int len);

/* Checkpoint.  The state buffer (host memory) is, in order, with no padding:
 *   uint64  magic 0x4146514D43535431, N, n_up, n_dn, K, W, P, step
 *           (K here counts the hidden variables of one sample: trial_slices x K)
 *   double  phi     W*N*(n_up+n_dn)*2  walker orbitals, column c < n_up spin up,
 *                                       column n_up + c spin down (re, im)
 *   double  weight  W
 *   double  x       W*P*K              hidden variables of the paths
 *   double  Phi     W*P*N*n_up         Phi(x_wp), kept so a resumed run is exact
 *                                       (complex, re im, for a trial other than alpha = 1, one slice)
 * afqmc_state_save with buf NULL stores the size in *len; otherwise *len must
 * be at least that size.  afqmc_state_load validates magic and shape.  The
 * random streams are counter based, so save + load + k steps is bitwise equal
 * to k steps without the interruption. */
afqmc_status afqmc_state_save(afqmc_ctx* ctx, void* buf, size_t* len);
afqmc_status afqmc_state_load(afqmc_ctx* ctx, const void* buf, size_t len);

/* Release the context (not the caller's workspace). */
void afqmc_destroy(afqmc_ctx* ctx);

/* Phase timing of afqmc_step with CUDA events on the context's stream
 * (recording does not synchronise).  afqmc_profile(ctx, 1) starts collecting,
 * afqmc_profile(ctx, 0) stops.  afqmc_profile_read synchronises and writes
 *   out[i]              milliseconds spent in phase i since the last read,
 *   out[AFQMC_PHASES+i] kernel launches of phase i,
 *   out[2*AFQMC_PHASES] steps profiled,
 * then resets.  Phases, in step order: 0 overlaps, LU and Theta at phi;
 * 1 fused contraction (force bias, local energy); 2 path-sign averages and the
 * mixed-estimator sums; 3 fields and the auxiliary-field matrices;
 * 4 propagation; 5 overlaps at phi' and ratios; 6 proposals and sum_k x_k U_k;
 * 7 trial orbitals exp(S) Phi0; 8 proposal overlaps; 9 acceptance;
 * 10 hand-off, re-orthonormalisation and bookkeeping; 11 population-control
 * comb (see pop_period); 12 error-controlled refinement of the tensor-core
 * contraction (see refine_tol; it runs right after phase 1). */
#define AFQMC_PHASES 13
afqmc_status afqmc_profile(afqmc_ctx* ctx, int enable);
afqmc_status afqmc_profile_read(afqmc_ctx* ctx, double* out, int len);

/* Number of CUDA kernels this library has launched in this process. */
int64_t afqmc_launch_count(void);

/* Which kernel computes the fused contraction of Eq. (15) and (27) for `cfg`:
 * 0 contract_fp64_kernel (precision FP64; when Theta does not fit in shared
 * memory, e.g. N = 200, it streams row slabs of Theta), 1 contract_tc_kernel (tensor cores,
 * per-pair form, N <= 128, n_up <= 32), 2 contract_tcy_kernel (tensor cores,
 * walker-side form B_p^T (L_g phi_w) with B_p = Phi_p A_p^-T, N <= 64 and
 * n_up + n_dn <= 40), 3 contract_fp64z_kernel (precision FP64, walker-side form
 * Phi_p^T (L_g phi_w) A_p^-1 for blocks of 8 or 16 pairs of a walker: when
 * n_paths >= 8 and the block's operands fit in shared memory, e.g. N <= 64),
 * 4 contract_fp64r_kernel (precision FP64 with rcache = 1: cached R_g,p Theta),
 * 5 contract_tcw_kernel (tensor cores, general walker-side form B_p^T (X_g phi_w),
 * N <= 256, n_up <= 64: see tc_form), 6 contract_fp64c_kernel (precision FP64 with
 * complex trial samples: R_g = Phi^dagger X_g);
 * -1 if `cfg` is NULL or no kernel supports its sizes.  Host only. */
int afqmc_contract_kernel(const afqmc_config* cfg);

/* Local energies, force-bias values and overlaps of a batch of (walker, trial
 * sample) pairs that allocates nothing.  The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc or give the library a workspace (code
 * inside another framework's operator hook whose device memory must come from
 * that framework's pool, or a loop where an allocation, which may synchronise the
 * device, is not allowed).  Its intermediate matrices live in one fixed device
 * array of afqmc_noalloc_scratch_bytes() bytes (32 MiB) that every GPU loading
 * the library holds until exit; the caller passes only inputs and outputs.
 *   h           N*N                      one-body matrix                    device
 *   L           n_chol*N*N               Cholesky vectors                   device
 *   Phi         n_pairs*N*n_up           trial orbitals of each pair        device
 *   phi         n_walkers*N*(n_up+n_dn)*2  walker orbitals (re, im; spin-up
 *                                        columns first); pair q uses walker
 *                                        q / pairs_per_walker              device
 *   logov       2*n_pairs   out: log <Phi_q|phi> (log|det| + i Arg det)    device
 *   e_local     2*n_pairs   out: local energy of each pair                 device
 *   force_bias  2*n_pairs*n_chol  out: <L_g> of each pair                  device
 * Runs asynchronously on `stream` on the calling thread's current device.
 * Returns AFQMC_ERR_ARG, without launching anything, when the batch needs more
 * than the fixed scratch (about n_pairs * (N*(n_up+n_dn)*16 + 32) bytes).
 * The first call on each device resolves the array's device address there
 * (cudaGetSymbolAddress) and caches it for the process; make that first call
 * before any stream capture.  The address is that of the device's primary
 * context (the runtime API's): calls from another driver-API context, or after
 * a cudaDeviceReset that follows the first call, are not supported.
 * Every call shares the array, so calls that overlap on the GPU race.  A
 * singular overlap gives log|ov| = -inf for that pair (its energy and force
 * bias are then those of a zero Theta; the other pairs are unaffected). */
size_t afqmc_noalloc_scratch_bytes(void);
afqmc_status afqmc_local_energy_noalloc(int N, int n_up, int n_dn, int n_chol, int64_t n_pairs,
                                        int pairs_per_walker, const double* h, const double* L,
                                        const double* Phi, const double* phi, double* logov,
                                        double* e_local, double* force_bias, void* stream);
/* Message of the last error of afqmc_local_energy_noalloc in this thread. */
const char* afqmc_noalloc_last_error(void);

/* Message of the last error in this thread (static storage). */
const char* afqmc_last_error(void);

/* Measured FP64 fused multiply-add rate of the current device (TFLOP/s, 2 flops
 * per FMA): a loop of independent register FMA chains over every SM, timed with
 * CUDA events on `stream`, best of three after a warm-up launch.  The peak the
 * FP64 path's contraction is compared with.  Synchronises. */
afqmc_status afqmc_fp64_fma_rate(double* tflops, void* stream);

/* Launch-shape autotuner: times the candidate shapes of the overlap kernel
 * (matrices per block), the tensor-core contraction (pairs per block) and the
 * trial-orbital kernel (threads per block) on this context's own data, keeps
 * the fastest, and caches the choice per problem shape for the process.
 * Results do not depend on the shapes.  Synchronises; not during capture.
 * chosen (nullable) receives the three choices (0 = built-in default). */
afqmc_status afqmc_autotune(afqmc_ctx* ctx, int* chosen);

/* The learned proposal (AFQMC_PROPOSAL_MLP), an extension the paper allows
 * (any proposal with an exact Metropolis acceptance, Sec. III A).  Walker
 * features f_k = Re sum_s Tr[(Phi0_s^T phi_s)^-1 Phi0_s^T U_k phi_s] (the gradient
 * of log|<Phi(x)|phi>| at x = 0); out = W3 tanh(W2 tanh(W1 f + b1) + b2) + b3 with
 * hidden width 256; mu = f + out[:K], logv = clip(out[K:], -6, 3).  GEMMs in BF16
 * with FP32 accumulation; master weights and Adam state FP32.  Parameters: one
 * flat float vector W1 (256 x K), b1 (256), W2 (256 x 256), b2 (256),
 * W3 (2K x 256), b3 (2K), row-major; afqmc_mlp_n_params(K) floats. */
int64_t afqmc_mlp_n_params(int K);
/* Copy the parameters out (set = 0) or in (set = 1); n must be afqmc_mlp_n_params(K). */
afqmc_status afqmc_mlp_params(afqmc_ctx* ctx, float* params, int64_t n, int set);
/* Evaluate the network on host inputs, for B <= n_walkers walkers:
 *   features B*K, x B*n_paths*K (hidden variables of the paths to fit),
 *   mu_logv (nullable) B*2K out: mu then logv per walker,
 *   loss (nullable) out: 1/(B P) sum 1/2 sum_k [(x - mu)^2/v + logv],
 *   grad (nullable) out: d loss / d params (flat layout).  Synchronises. */
afqmc_status afqmc_mlp_eval(afqmc_ctx* ctx, int B, const float* features, const double* x, float* mu_logv,
                            double* loss, float* grad);
/* Features, mu and logv (each n_walkers*K floats, nullable) the last step used. */
afqmc_status afqmc_mlp_state(afqmc_ctx* ctx, float* features, float* mu, float* logv);

/* Several systems (contexts of any sizes and precisions) stepped together: one
 * leapfrog step of every context is captured once into one CUDA graph (a fork
 * on `stream`, each context's kernels as a branch on its own stream, a join),
 * and each afqmc_batch_step launches that graph once per step.  The contexts that
 * use the walker-side tensor-core contraction with one operand arithmetic (the
 * first such context's; their Y images in one chunk of walkers) share its dominant
 * kernel: their branches stop after the contraction's images, one persistent
 * launch on `stream` runs every such system's GEMM-Z blocks from one list, and
 * their branches resume (the results are the same bit for bit).  Every context
 * needs its own non-default stream, distinct from `stream`; the contexts stay
 * usable one by one (afqmc_energy, save/load, ...) between batch steps after
 * afqmc_batch_sync.  The batch does not own the contexts. */
typedef struct afqmc_batch afqmc_batch;
afqmc_status afqmc_batch_create(int n_systems, afqmc_ctx* const* ctxs, void* stream, afqmc_batch** out);
afqmc_status afqmc_batch_step(afqmc_batch* batch, int n_steps);  /* asynchronous on `stream` */
afqmc_status afqmc_batch_sync(afqmc_batch* batch);
/* How many of the batch's systems share the one GEMM-Z launch (-1 for NULL). */
int afqmc_batch_shared_contractions(const afqmc_batch* batch);
void afqmc_batch_destroy(afqmc_batch* batch);

/* The library's Philox4x32-10 (Salmon et al., SC'11) on the device, for
 * checking the generator: out[4*i + j] = word j of Philox(counter_i, key) with
 * counter_i = {c0 + i, c1, c2, c3}, i < n.  out is a device pointer. */
afqmc_status afqmc_philox_fill(uint32_t* out, int64_t n, uint32_t c0, uint32_t c1, uint32_t c2,
                               uint32_t c3, uint64_t key, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AFQMC_H */
