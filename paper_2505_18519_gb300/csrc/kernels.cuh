// Declarations of the library's kernels and their host launchers.
#pragma once
#include "common.cuh"

// api.cu: record an error message for afqmc_last_error and return `st`
afqmc_status set_error(afqmc_status st, const char* fmt, ...);
// api.cu: one step of a context in a batch whose walker-side GEMM-Z runs in one
// launch for all systems: part 1 up to the contraction's images, part 2 the rest.
namespace afq {
afqmc_status batch_step_part(afqmc_ctx* ctx, int part);
}
// api.cu: the tensor-core form of a mixed-precision configuration (the value
// afqmc_contract_kernel reports: 1 per-pair, 2 walker-side for N <= 64,
// 5 general walker-side), -1 if the chosen form does not support its sizes.
int tc_kind(const afqmc_config* c);

namespace afq {

// linalg_fp64.cu
void gemm_nn_f64(cudaStream_t s, int M, int Nc, int K, double alpha, const double* A, long long lda, const double* B,
                 long long ldb, double beta, double* C, long long ldc);
enum OverlapOutput { OVL_THETA = 0, OVL_TRIAL = 1, OVL_INVERSE = 2 };
// th2 (nullable, with Theta): ||A^-1||_F^2 per pair and spin at th2[2 pair + spin]
// (infinite for a singular or non-finite overlap).  list, n_list (nullable): only
// the pairs list[0 .. *n_list), a device list, with the grid sized for `pairs` of them.
// PhiD, phiD (nullable; the mixed-precision path, real trial, n <= 64): double-float
// copies of Phi (same strides, 8 bytes per entry) and of the walkers (16 bytes per
// complex entry, from u_to_df of the FP64 arrays): A = Phi^T phi is then formed
// in double-float (compensated sums), the LU, log det and A^-1 stay FP64.  b_df
// (with PhiD and OVL_TRIAL): B = Phi A^-T in double-float, written as (Re hi, Re
// lo, Im hi, Im lo) per entry in place of the FP64 values.  Apre (nullable): A of
// every pair already formed (overlap_tc; n x n entries per pair, row-major, as
// double-float (Re hi, Re lo, Im hi, Im lo)), read instead of the products.
cudaError_t overlap_lu(cudaStream_t s, const Dims& d, int spin, const double* Phi, long long Phi_stride,
                       const double2* phi, double2* logdet, double2* Theta, const int* alive, int* status,
                       long long pairs, int P, int trial_side = OVL_THETA, double* th2 = nullptr,
                       const int* list = nullptr, const int* n_list = nullptr, const void* PhiD = nullptr,
                       const void* phiD = nullptr, bool b_df = false, const void* Apre = nullptr);
// Both spins: one warp per pair (half a warp per spin) when n_up <= 16 and no
// double-float products are asked for, else overlap_lu for each spin.  Same results.
// Apre: both spins' A from overlap_tc (spin down at offset d.pairs n_up^2 entries).
cudaError_t overlap_lu_both(cudaStream_t s, const Dims& d, const double* Phi, long long Phi_stride,
                            const double2* phi, double2* logdet, double2* Theta, const int* alive, int* status,
                            long long pairs, int P, int trial_side = OVL_THETA, double* th2 = nullptr,
                            const void* PhiD = nullptr, const void* phiD = nullptr, bool b_df = false,
                            const void* Apre = nullptr);
// overlap_tc.cu: A_p = Phi_p^T phi_w of every pair and spin on the tensor cores
// (exact 8-bit digit products, about 40 bits) from the double-float copies PhiD,
// phiD of the mixed-precision path, real trial, N <= 128, n <= 40 per spin;
// written to Aout (d.pairs (n_up^2 + n_dn^2) entries of 16 bytes) for overlap_lu.
// Pairs of walkers with alive[w] == 0 are skipped (alive nullable).
bool overlap_tc_supported(int N, int n);
// overlap_lu_df.cu: the LU, log det A and (with Theta) A^-1, ||A^-1||_F^2 (th2) and
// B = Phi A^-T (double-float, OVL_TRIAL layout) of one spin from the tensor-core
// A (Apre of that spin), in double-float arithmetic on the FP32 pipe; overlap_lu
// hands its calls with Apre to it.
cudaError_t overlap_lu_df(cudaStream_t s, const Dims& d, int spin, const void* Apre, double2* logdet, double2* Theta,
                          const int* alive, int* status, long long pairs, int P, double* th2, const void* PhiD,
                          long long Phi_stride);
cudaError_t overlap_tc(cudaStream_t s, const Dims& d, const void* PhiD, long long Phi_stride, const void* phiD,
                       const int* alive, void* Aout, int* status);
cudaError_t reorthonormalise(cudaStream_t s, const Dims& d, const double2* src, double2* dst, const int* alive,
                             int* status, int n_walkers);
// Phi = exp(S) Phi0 for `problems` symmetric S (FP64).  trial_orbitals runs the
// Chebyshev series on a Lanczos-estimated spectral interval with an a-posteriori
// check (trial_df.cu); trial_orbitals_gershgorin on the Gershgorin interval of S
// (linalg_fp64.cu), also the fallback when S does not fit in shared memory.
cudaError_t trial_orbitals(cudaStream_t s, int N, int nu, long long problems, const double* S_all, const double* Phi0,
                           double* Out, const int* alive, int P, int* status, int threads = 256);
cudaError_t trial_orbitals_gershgorin(cudaStream_t s, int N, int nu, long long problems, const double* S_all,
                                      const double* Phi0, double* Out, const int* alive, int P, int* status,
                                      int threads = 256);
// trial_df.cu: the same in double-float arithmetic (mixed-precision path); S_all
// is scratch (converted in place when S does not fit in shared memory)
cudaError_t trial_orbitals_df(cudaStream_t s, int N, int nu, long long problems, double* S_all, const double* Phi0,
                              double* Out, const int* alive, int P, int* status, int threads = 256,
                              bool s_is_df = false);
bool trial_orbitals_df_supported(int N, int nu);
// With S as double-float pairs and too large for shared memory, the same kernel
// reads S from global memory: N <= 256 and 3 N n_up doubles of vectors in 200 KB.
bool trial_orbitals_dfg_supported(int N, int nu);
// The double-float kernel for the problems list[0 .. *count) (a device list), on
// one block per SM.
cudaError_t trial_orbitals_df_list(cudaStream_t s, int N, int nu, const double* S_all, bool s_is_df, const double* Phi0,
                                   double* Out, const int* alive, int P, int* status, const int* list,
                                   const int* count);
// trial_tc.cu: the same series with the products S V on the tensor cores (8-bit
// digit splitting, exact integer accumulation, about 40 bits per product);
// N <= 128, n_up <= 32.  Problems whose Chebyshev vectors grow (the Lanczos
// interval missed part of the spectrum) are listed in redo_list / *redo_count
// (workspace of `problems` + 1 ints) and redone by the double-float kernel.
// lim: polls of an mbarrier wait before it gives up (0: 2^26).
bool trial_orbitals_tc_supported(int N, int nu);
// sprop_tc.cu: S = X U (M rows of X, K <= 128 variables, NN = N^2 columns) on the
// tensor cores as exact 8-bit digit products (about 40 bits), written as
// double-float pairs (8 bytes per entry) like gemm_df; img holds U's digit images
// and column exponents (sprop_u_image_bytes, formed once by sprop_u_images).
bool sprop_tc_supported(int K, long long NN);
size_t sprop_u_image_bytes(int K, long long NN);
cudaError_t sprop_u_images(cudaStream_t s, int K, long long NN, const double* U, void* img);
cudaError_t sprop_tc(cudaStream_t s, long long M, int K, long long NN, const double* X, const void* img, void* S,
                     int* status, uint32_t lim);
size_t trial_orbitals_tc_smem(int nu);
// counters[9] += the terms of every finished problem, counters[10] += the problems redone.
cudaError_t trial_orbitals_tc(cudaStream_t s, int N, int nu, long long problems, const double* S_all, bool s_is_df,
                              const double* Phi0, double* Out, const int* alive, int P, int* status, int* redo_list,
                              int* redo_count, unsigned long long* counters, uint32_t lim);
// S = X U in double-float (X FP64 M x K, U as double-float K x Nc from u_to_df);
// S is written as double-float pairs, 8 bytes per element
cudaError_t u_to_df(cudaStream_t s, long long n, const double* U, void* Ud);
// Xdf (optional): M*K*8 bytes of work space to hold X in double-float, formed
// once instead of once per column tile of S.
cudaError_t gemm_df(cudaStream_t s, int M, int Nc, int K, const double* X, const void* Ud, double* S,
                    void* Xdf = nullptr);
cudaError_t one_body_propagator(cudaStream_t s, int N, int G, double dtau, const double* h, const double* L, double* T,
                                double* scratch3, double* expT);

// contract_fp64.cu
cudaError_t contract_fp64(cudaStream_t s, const Dims& d, const double* h, const double* L, const double* Phi,
                          const double2* Theta, double2* vpair, double2* epair, long long pairs);
bool contract_fp64_supported(int N, int nu, int nd);
// Error-controlled refinement of the tensor-core contraction (per-pair form):
// lam = sum_g ||L_g||_2^2 (lam_g: G scratch values), once at init; per
// measurement, the pairs each walker must recompute in FP64 so that its
// estimated error stays below tol, appended to items (count in *n_items,
// cumulative count in counters[5]).
cudaError_t refine_scale(cudaStream_t s, int N, int G, const double* L, double* lam_g, double* lam);
// th2_spins (nullable): ||Theta_p||_F^2 per pair and spin from the overlap kernel,
// used instead of forming ||Theta_p||_F^2 from Theta; u: the contraction's
// resolution in the error model (2^-20 for the per-pair form).
cudaError_t refine_select(cudaStream_t s, const Dims& d, double tol, const double* lam, const double2* logdet,
                          const double2* Theta, double* th2, const int* alive, int* items, int* n_items,
                          unsigned long long* counters, const double* th2_spins = nullptr, double u = 0x1p-20);
// The same contraction for the pairs items[0 .. *n_items) only (a device list of
// pair indices, *n_items <= max_items), the others' vpair/epair left as they are;
// with hdf and Ldf (double-float copies of h and L from u_to_df) R and M run in
// double-float arithmetic instead of FP64 (about 44 bits).
cudaError_t contract_fp64_listed(cudaStream_t s, const Dims& d, const double* h, const double* L, const double* Phi,
                                 const double2* Theta, double2* vpair, double2* epair, const int* items,
                                 const int* n_items, long long max_items, const void* hdf = nullptr,
                                 const void* Ldf = nullptr, void* part = nullptr, long long part_cap = 0);
// (part, part_cap: with the double-float copies, space for part_cap double2 partial
// sums; each listed pair's matrices are then split into up to 16 runs, one block
// each, and the runs' sums added in order: a few listed pairs fill the GPU.)
// Walker-side FP64 form (Y_g = X_g phi_w once per block of a walker's pairs,
// Z = Phi_p^T Y_g, Q = Z A_p^-1; Tr Q and Tr Q^2 are those of M_g): needs A^-1
// per pair and spin (overlap_lu with OVL_INVERSE) and the walkers.
bool contract_fp64_walker_side(int N, int nu, int nd, int P);
// L must follow h directly ([h; L] one (G+1) N x N matrix); work: W (G+1) N 2nt
// + N W 2nt doubles (contract_fp64_walker_bytes), where Y_g = X_g phi_w of every
// walker is formed by one GEMM before the contraction reads it.
size_t contract_fp64_walker_bytes(int N, int nu, int nd, int G, long long W, int P);
cudaError_t contract_fp64_walker(cudaStream_t s, const Dims& d, const double* h, const double* L, const double* Phi,
                                 const double2* Ainv, const double2* phi, void* work, double2* vpair, double2* epair);

// contract_tc.cu
bool contract_tc_supported(int N, int nu, int nd, bool f16);
size_t contract_tc_image_bytes(int N, int nu, int nd, int G, bool f16);
cudaError_t contract_tc_prepare(cudaStream_t st, int N, int nu, int nd, int G, const double* h, const double* L,
                                void* image, bool f16);
// With contract_tc_walker_side(...) true the contraction takes B = Phi A^-T per
// pair (overlap_lu with trial_side = true) in place of Theta, plus the walkers.
bool contract_tc_walker_side(int N, int nu, int nd, bool f16);
// Work space of the walker-side form: the split images of Y_g = X_g phi_w of
// every walker and their scale exponents (0 when the form does not apply).
size_t contract_tcy_yimage_bytes(int N, int nu, int nd, int G, long long W, bool f16);
cudaError_t contract_tc(cudaStream_t st, const Dims& d, const void* image, const double* Phi, const double2* Theta,
                        const double2* phi, void* ywork, double2* vpair, double2* epair, int* status, bool f16);

// contract_tcw.cu: the walker-side tensor-core form for any size of the FP64
// path (N <= 256, n_up <= 64): Z_{p,g} = B_p^T (X_g phi_w), B_p = Phi_p A_p^-T from
// overlap_lu with OVL_TRIAL.  work: contract_tcw_work_bytes bytes (the split
// image of X_g, per chunk of walkers the images of Y_g and B_p, per-pair traces);
// contract_tcw_prepare fills the X image once (h and L must not change after).
// mode: operand arithmetic, 0 bf16x3, 1 fp16x3, 2 fp16x6 (tc_mode of the config).
bool contract_tcw_supported(int N, int nu, int nd, int G, long long W, int P, int mode);
size_t contract_tcw_work_bytes(int N, int nu, int nd, int G, long long W, int P, int mode);
cudaError_t contract_tcw_prepare(cudaStream_t st, const Dims& d, const double* h, const double* L, void* work,
                                 int mode);
// b_df: Bm holds B as double-float pairs (overlap_lu with b_df), else FP64.
cudaError_t contract_tcw(cudaStream_t st, const Dims& d, void* work, const double2* Bm, const double2* phi,
                         double2* vpair, double2* epair, int* status, int mode, bool b_df = false);
// The same in three parts, for a context whose Y images of both spins fit one chunk
// of walkers side by side (contract_tcw_single_chunk): the images of both spins
// (contract_tcw_images), then GEMM-Z, here
// described per spin (contract_tcw_zargs; n == 0 for an empty spin) so that a batch
// of systems runs it in one launch (contract_tcw_multi), then the per-pair finish.
struct TcwZArgs {
    int n, G1, KZ, KC, NT, GB, NTILES, P, PB, MT, S, a_res;
    long long w0, blocks;         // first walker of the work; blocks (walkers x pair tiles)
    const uint8_t* Aimg;
    const int* aexp;
    const uint8_t* Yimg;
    const int* yexp;
    float2* vpart;
    double2* exsum;
    int* status;
    size_t smem;                  // dynamic shared memory a block needs
};
constexpr int TCWZ_MAXWORK = 32;
struct TcwZMulti {
    int n;                                  // pieces of work
    long long first[TCWZ_MAXWORK + 1];      // first block of each piece; first[n] = total
    TcwZArgs a[TCWZ_MAXWORK];
};
bool contract_tcw_single_chunk(const Dims& d, int mode);
cudaError_t contract_tcw_images(cudaStream_t st, const Dims& d, void* work, const double2* Bm, const double2* phi,
                                int* status, int mode, bool b_df);
bool contract_tcw_zargs(const Dims& d, void* work, int* status, int mode, int spin, TcwZArgs* out);
cudaError_t contract_tcw_multi(cudaStream_t st, const TcwZMulti& m, int mode, uint32_t lim);
cudaError_t contract_tcw_finish(cudaStream_t st, const Dims& d, void* work, double2* vpair, double2* epair, int mode);

// trial_complex.cu: complex and multi-slice trial samples (FP64 path).
// Out = exp(alpha S) V0 per problem (S real symmetric in S_all; V0 = the real
// Phi0 when Vin is NULL, else Vin[problem], complex); Chebyshev series of
// complex coefficients on the Gershgorin interval.
bool trial_orbitals_c_supported(int N, int nu);
cudaError_t trial_orbitals_c(cudaStream_t s, int N, int nu, long long problems, const double* S_all, double2 alpha,
                             const double* Phi0, const double2* Vin, double2* Out, const int* alive, int P,
                             int* status);
// Out[problem] = Pm V[problem] (the fixed propagator between slices).
cudaError_t slice_propagate(cudaStream_t s, int N, int nu, long long problems, const double* Pm, const double2* V,
                            double2* Out, const int* alive, int P);
cudaError_t walkers_from_trial_c(cudaStream_t s, const Dims& d, const double2* Phi_w, double2* phi);
// The per-pair FP64 contraction with complex Phi (R_g = Phi^dagger X_g); with
// list, n_list (device) only the pairs list[0 .. *n_list).
bool contract_fp64c_supported(int N, int nu, int nd);
cudaError_t contract_fp64c(cudaStream_t s, const Dims& d, const double* h, const double* L, const double2* Phi,
                           const double2* Theta, double2* vpair, double2* epair, const int* list = nullptr,
                           const int* n_list = nullptr);

// walker.cu
struct StepParams {
    uint64_t seed;
    long long woff;   // global index of walker 0
    double dtau, pcn_beta, e_shift, kill_threshold, rw_step, mlp_mix;
    int constraint, proposal, taylor_order, history_capacity;
    int importance, pop_period;
};
cudaError_t fill_normals(cudaStream_t s, double* out, long long rows, int cols, long long entity0, uint64_t seed,
                         uint32_t tag, const unsigned long long* step_ctr, uint32_t sweep);
cudaError_t walkers_from_trial(cudaStream_t s, const Dims& d, const double* Phi_w, double2* phi);
cudaError_t walker_average(cudaStream_t s, const Dims& d, const double2* logdet, const double2* vpair,
                           const double2* epair, double2* logov, double2* sumS, double2* vbar, double2* ebar);
cudaError_t energy_reduce(cudaStream_t s, const Dims& d, const double* weight, const double2* ebar,
                          const double2* sumS, double* out3);
cudaError_t fields(cudaStream_t s, const Dims& d, const StepParams& p, const unsigned long long* ctr,
                   const double2* vbar, const double2* sumS, double* weight, int* alive, double* yplanes,
                   double2* logshift);
// scratch: W * 2 * N * nt complex work space, used (and then required) only when
// propagate_in_smem(N, nt) is false.
bool propagate_in_smem(int N, int nt);
cudaError_t propagate(cudaStream_t s, const Dims& d, const StepParams& p, const double* expT, const double* Aplanes,
                      const double2* phi, double2* phi_new, const int* alive, double2* scratch);
// The same propagation with expT and the field planes as double-float (from
// u_to_df and gemm_df), for the mixed-precision path; needs propagate_in_smem.
cudaError_t propagate_df(cudaStream_t s, const Dims& d, const StepParams& p, const void* expTdf, const void* Aplanes_df,
                         const double2* phi, double2* phi_new, const int* alive);
cudaError_t ratios(cudaStream_t s, const Dims& d, const double2* logov, const double2* logdet_new,
                   const double2* sumS, const double2* logshift, const int* alive, double2* logov_cur,
                   double2* old_sum, double2* ratio, double* Iabs);
cudaError_t propose(cudaStream_t s, const Dims& d, const StepParams& p, const unsigned long long* ctr, uint32_t tag,
                    uint32_t tag_acc, uint32_t sweep, const double* x, const int* alive, const float* mu,
                    const float* logv, double* xprop);
cudaError_t accept(cudaStream_t s, const Dims& d, const StepParams& p, const unsigned long long* ctr, uint32_t tag,
                   uint32_t sweep, const double2* logdet_prop, const double* xprop, const double* Phiprop,
                   const int* alive, const float* mu, const float* logv, double2* logov_cur, double* x, double* Phi,
                   unsigned long long* counters, int* rdirty = nullptr);
cudaError_t combine_logdet(cudaStream_t s, long long pairs, const double2* logdet, double2* logov);
cudaError_t handoff(cudaStream_t s, const Dims& d, const StepParams& p, const double2* logov_cur,
                    const double2* old_sum, const double2* ratio, const double* Iabs, const double2* ebar,
                    const int* alive, double* weight, int* status);
// Extra measurement paths: the walkers that count, the per-walker sums over a
// round's paths (acc: 2W), and the estimate (out: 2W + 2, see walker.cu).
cudaError_t meas_alive(cudaStream_t s, const Dims& d, double thr, const double* weight, const double2* sumS,
                       int* alive);
cudaError_t meas_accumulate(cudaStream_t s, const Dims& d, const double2* logov, const double2* epair,
                            const int* alive, double2* acc);
cudaError_t meas_finish(cudaStream_t s, const Dims& d, int rounds, const double* weight, const double2* sumS0,
                        const int* alive, const double2* acc, double2* out);
// rcache.cu: half-rotated matrices (X_g Phi_p) cached per pair, refreshed for the
// pairs flagged dirty, and the FP64 contraction that reads them.
bool contract_fp64r_supported(int N, int nu, int nd);
size_t rcache_bytes(int N, int nu, int G, long long pairs);
cudaError_t rcache_refresh(cudaStream_t s, const Dims& d, const double* X, const double* Phi, int* dirty, int* list,
                           int* count, double* Rc, unsigned long long* counters);
cudaError_t contract_fp64r(cudaStream_t s, const Dims& d, const double* Rc, const double2* Theta, double2* vpair,
                           double2* epair);
// Comb population control after every p.pop_period-th step (decided on the
// device from counters[0]), gathering the walker state in place; cum, hit,
// slot and from are W entries of scratch each, flag two ints.
// The cached half-rotated matrices Rc and their dirty flags (both nullable) move
// with the walkers.
cudaError_t population_control(cudaStream_t s, const Dims& d, const StepParams& p, unsigned long long* counters,
                               double* weight, double2* phi, double* x, double* Phi, double* Rc, int* rdirty,
                               double* cum, int* hit, int* slot, int* from, int* flag);
cudaError_t step_end(cudaStream_t s, const StepParams& p, const double* measured3, double* history,
                     unsigned long long* counters);
cudaError_t set_value(cudaStream_t s, double* out, long long n, double v);

// mlp.cu
long long mlp_n_params(int K);
cudaError_t mlp_prepare(cudaStream_t s, const Dims& d, const MlpBuffers& m, const double* U, const double* Phi0,
                        uint64_t seed);
cudaError_t mlp_pack(cudaStream_t s, const Dims& d, const MlpBuffers& m);
cudaError_t mlp_features(cudaStream_t s, const Dims& d, const MlpBuffers& m, const double* Phi0, const double2* phi,
                         int* status);
cudaError_t mlp_forward(cudaStream_t s, const Dims& d, const MlpBuffers& m, int rows);
cudaError_t mlp_backward(cudaStream_t s, const Dims& d, const MlpBuffers& m, int rows, const double* x, float lr,
                         bool apply);
cudaError_t set_int(cudaStream_t s, int* out, long long n, int v);

}  // namespace afq
