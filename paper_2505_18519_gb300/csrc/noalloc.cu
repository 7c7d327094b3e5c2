// Local energies and force-bias values of a batch of (walker, trial sample)
// pairs with no device allocation at all: the intermediate Theta matrices and
// per-spin log-determinants live in one file-scope device array instead of a
// caller-provided workspace.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// embedded in another framework's custom-operator hook, where device memory may
// only come from that framework's own pool, and latency-critical loops where an
// allocation (which can synchronise the device) is not allowed.  They pass only
// their inputs and outputs.
//
// The array is shared by every call in the process, on every device that loads
// the library, and keeps the last call's contents.  Only its status word must
// start at zero, and each call clears it; every other element a call reads is
// first written by that same call.  Calls that overlap on the GPU (other
// streams, other host threads, the same device) race on it.
#include <stdio.h>

#include <mutex>

#include "kernels.cuh"

using namespace afq;

// 32 MiB of scratch, resident on every GPU that loads the library until exit.
static constexpr size_t kNoallocScratchBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256];   // device address of the array, per device ordinal

static thread_local char g_noalloc_err[256] = "";

static afqmc_status noalloc_fail(afqmc_status st, const char* msg, cudaError_t e = cudaSuccess) {
    if (e != cudaSuccess)
        snprintf(g_noalloc_err, sizeof g_noalloc_err, "%s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(g_noalloc_err, sizeof g_noalloc_err, "%s", msg);
    return st;
}

extern "C" const char* afqmc_noalloc_last_error(void) { return g_noalloc_err; }

extern "C" size_t afqmc_noalloc_scratch_bytes(void) { return kNoallocScratchBytes; }

extern "C" afqmc_status afqmc_local_energy_noalloc(int N, int n_up, int n_dn, int n_chol, int64_t n_pairs,
                                                   int pairs_per_walker, const double* h, const double* L,
                                                   const double* Phi, const double* phi, double* logov,
                                                   double* e_local, double* force_bias, void* stream) {
    if (N < 1 || N > 256 || n_up < 1 || n_up > N || n_up > 64 || n_dn < 0 || n_dn > n_up || n_chol < 1 ||
        n_pairs < 0 || pairs_per_walker < 1)
        return noalloc_fail(AFQMC_ERR_ARG, "invalid sizes");
    if (!h || !L || !Phi || !phi || !logov || !e_local || !force_bias)
        return noalloc_fail(AFQMC_ERR_ARG, "every array must be a device pointer (none may be NULL)");
    if (!contract_fp64_supported(N, n_up, n_dn))
        return noalloc_fail(AFQMC_ERR_ARG, "sizes too large for the FP64 contraction kernel");
    const int nt = n_up + n_dn;
    // Bound n_pairs before any product with it, so that no size below can wrap: every
    // pair takes N nt complex Theta entries and two complex log-determinants, and the
    // layout adds at most 255 bytes of alignment and the status word.
    const size_t per_pair = (size_t)N * nt * sizeof(double2) + 2 * sizeof(double2);
    const size_t fixed = 256 + sizeof(int);
    if (n_pairs > 0 && (uint64_t)n_pairs > (kNoallocScratchBytes - fixed) / per_pair) {
        snprintf(g_noalloc_err, sizeof g_noalloc_err,
                 "batch of %lld pairs needs more scratch than the fixed maximum of %zu bytes "
                 "(about n_pairs * (N * (n_up + n_dn) * 16 + 32)); split the batch",
                 (long long)n_pairs, kNoallocScratchBytes);
        return AFQMC_ERR_ARG;
    }
    if ((n_pairs + pairs_per_walker - 1) / pairs_per_walker > INT32_MAX)
        return noalloc_fail(AFQMC_ERR_ARG, "too many walkers in the batch");
    const size_t theta_bytes = (size_t)n_pairs * N * nt * sizeof(double2);
    const size_t logdet_off = (theta_bytes + 255) & ~(size_t)255;
    const size_t status_off = logdet_off + (size_t)n_pairs * 2 * sizeof(double2);
    if (n_pairs == 0) return AFQMC_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(AFQMC_ERR_CUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= 256) return noalloc_fail(AFQMC_ERR_ARG, "device ordinal out of range");
    void* base = nullptr;
    {
        // Set-up, once per device, with that device current: the host-side name
        // of the array is not a device address, so ask the runtime for it.  The
        // address belongs to the device's primary context (the one the runtime
        // API uses); it is cached for the life of the process, so neither another
        // driver-API context made current nor a cudaDeviceReset after this first
        // call is supported.
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return noalloc_fail(AFQMC_ERR_CUDA, "cudaGetSymbolAddress", e);
            g_noalloc_addr[dev] = p;
        }
        base = g_noalloc_addr[dev];
    }
    double2* Theta = reinterpret_cast<double2*>(base);
    double2* logdet = reinterpret_cast<double2*>(static_cast<char*>(base) + logdet_off);
    cudaStream_t s = (cudaStream_t)stream;
    Dims d{};   // value-initialised: launch shapes at their defaults
    d.N = N; d.nu = n_up; d.nd = n_dn; d.nt = nt; d.G = n_chol; d.K = 1;
    d.P = pairs_per_walker;
    d.W = (int)((n_pairs + pairs_per_walker - 1) / pairs_per_walker);
    d.pairs = n_pairs;
    // the overlap kernel flags singular overlaps in a status word, which lives in
    // the scratch too and is cleared first (a singular pair gets log|ov| = -inf)
    int* status = reinterpret_cast<int*>(static_cast<char*>(base) + status_off);
    e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e != cudaSuccess) return noalloc_fail(AFQMC_ERR_CUDA, "clearing the status word", e);
    for (int spin = 0; spin < 2; ++spin) {
        e = overlap_lu(s, d, spin, Phi, (long long)N * n_up, reinterpret_cast<const double2*>(phi), logdet, Theta,
                       nullptr, status, n_pairs, pairs_per_walker);
        if (e != cudaSuccess) return noalloc_fail(AFQMC_ERR_CUDA, "overlap kernel", e);
    }
    e = contract_fp64(s, d, h, L, Phi, Theta, reinterpret_cast<double2*>(force_bias), reinterpret_cast<double2*>(e_local),
                      n_pairs);
    if (e != cudaSuccess) return noalloc_fail(AFQMC_ERR_CUDA, "contraction kernel", e);
    e = combine_logdet(s, n_pairs, logdet, reinterpret_cast<double2*>(logov));
    if (e != cudaSuccess) return noalloc_fail(AFQMC_ERR_CUDA, "log-determinant kernel", e);
    return AFQMC_OK;
}
