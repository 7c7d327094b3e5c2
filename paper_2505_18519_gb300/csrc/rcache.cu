// Half-rotated matrices cached per pair, and the FP64 contraction that reads
// them.
//
// For pair p with trial orbitals Phi_p (N x n_up, real) the matrices
//   R_g,p = Phi_p^T X_g   (n_up x N;  X_0 = h, X_g+1 = L_g)
// depend on the path only, not on the walker, so they change only when a
// Metropolis move of the path is accepted (Eq. (23)).  Kept from one step to
// the next they turn the contraction into
//   M_g,s = R_g,p[:n_s] Theta_s,   Theta_s = phi_s A_s^-1   (Eq. (27)),
// 2 N (n_up^2 + n_dn^2) FP64 multiply-adds per pair and matrix, against
// 2 N (n_up^2 + n_dn^2) + 4 (n_up^3 + n_dn^3) + 2 N^2 (n_up + n_dn) / P for the
// walker-side form; each measurement first refreshes the pairs whose path
// moved since the last one (n_up N^2 multiply-adds per matrix and pair).
//
// Storage: Rc[pair][g1][k][a] = (X_g1 Phi_p)[k, a] = R_g1,p[a, k] (X symmetric),
// (G + 1) N n_up doubles per pair.  dirty[pair] = 1 marks a pair to refresh.
#include "kernels.cuh"

namespace afq {

constexpr int RC_T = 256;        // threads per block of the refresh
constexpr int RC_PAIRS = 8;      // pairs per work item of the refresh
constexpr int RC_GCHUNK = 16;    // matrices per work item of the refresh
constexpr int CR_MAXWARPS = 8;   // warps (pairs) per block of the contraction
constexpr int CR_MINWARPS = 4;

// Appends every dirty pair to list (in no particular order) and clears its flag.
__global__ void rcache_collect_kernel(long long pairs, int* __restrict__ dirty, int* __restrict__ list, int* count) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= pairs || !dirty[p]) return;
    dirty[p] = 0;
    list[atomicAdd(count, 1)] = (int)p;
}

// Work item (c, gc): listed pairs c RC_PAIRS .. + RC_PAIRS - 1 and matrices
// gc RC_GCHUNK .. + RC_GCHUNK - 1.  Phi of the item's pairs and one X_g at a
// time sit in shared memory; each thread forms whole output entries.
__global__ void __launch_bounds__(RC_T) rcache_fill_kernel(int N, int nu, int G, const double* __restrict__ X,
                                                          const double* __restrict__ Phi, const int* __restrict__ list,
                                                          const int* __restrict__ count, double* __restrict__ Rc) {
    extern __shared__ double srf[];
    const int Nnu = N * nu;
    double* sX = srf;                            // N x N
    double* sPh = srf + (size_t)N * N;           // RC_PAIRS x N x nu
    const long long n = *count;
    const long long chunks = (n + RC_PAIRS - 1) / RC_PAIRS;
    const int gchunks = (G + 1 + RC_GCHUNK - 1) / RC_GCHUNK;
    const long long per_pair = (long long)(G + 1) * Nnu;
    for (long long it = blockIdx.x; it < chunks * gchunks; it += gridDim.x) {
        const long long c = it / gchunks;
        const int g0 = (int)(it - c * gchunks) * RC_GCHUNK;
        const int g1 = min(G + 1, g0 + RC_GCHUNK);
        const int np = (int)min((long long)RC_PAIRS, n - c * RC_PAIRS);
        for (int e = threadIdx.x; e < np * Nnu; e += RC_T) {
            const int q = e / Nnu;
            sPh[e] = Phi[(long long)list[c * RC_PAIRS + q] * Nnu + (e - q * Nnu)];
        }
        for (int g = g0; g < g1; ++g) {
            const double* Xg = X + (long long)g * N * N;
            for (int e = threadIdx.x; e < N * N; e += RC_T) sX[e] = Xg[e];
            __syncthreads();
            for (int o = threadIdx.x; o < np * Nnu; o += RC_T) {
                const int q = o / Nnu, r = o - q * Nnu, k = r / nu, a = r - k * nu;
                const double* xr = sX + (size_t)k * N;
                const double* pc = sPh + (size_t)q * Nnu + a;
                double acc = 0.0;
                for (int j = 0; j < N; ++j) acc = fma(xr[j], pc[(size_t)j * nu], acc);
                Rc[(long long)list[c * RC_PAIRS + q] * per_pair + (long long)g * Nnu + r] = acc;
            }
            __syncthreads();   // sX is overwritten next; sPh next item
        }
    }
}

static size_t rcache_fill_smem(int N, int nu) { return ((size_t)N * N + (size_t)RC_PAIRS * N * nu) * sizeof(double); }

// Per-warp shared memory of the contraction: Theta (N x nt complex), one R_g
// (N x n_up), M of both spins (n_up^2 + n_dn^2 complex).
__host__ __device__ __forceinline__ size_t contract_fp64r_warp_bytes(int N, int nu, int nd) {
    const size_t nt = nu + nd;
    return (2 * (size_t)N * nt + ((size_t)N * nu + 1) / 2 * 2 + 2 * ((size_t)nu * nu + (size_t)nd * nd)) *
           sizeof(double);
}

static int contract_fp64r_warps(int N, int nu, int nd) {
    const size_t per = contract_fp64r_warp_bytes(N, nu, nd);
    int w = (int)((size_t)(220 * 1024) / per);
    return w > CR_MAXWARPS ? CR_MAXWARPS : w;
}

bool contract_fp64r_supported(int N, int nu, int nd) {
    if (N < 1 || nu < 1 || nd < 0 || nd > nu || nu > 64) return false;
    return contract_fp64r_warps(N, nu, nd) >= CR_MINWARPS && rcache_fill_smem(N, nu) <= 200 * 1024;
}

size_t rcache_bytes(int N, int nu, int G, long long pairs) {
    return (size_t)pairs * (size_t)(G + 1) * (size_t)N * (size_t)nu * sizeof(double);
}

// One warp per pair: Theta stays in the warp's shared memory; per matrix the
// warp loads its R_g, forms the n_up^2 + n_dn^2 entries of M of both spins
// (lane-strided, each a full k-sum: splitting the sums over lanes would cost
// FP64 additions, which take the same pipe as the multiply-adds), then sums
// Tr M and Tr M^2 by shuffles.  No block-wide barrier: warps run independently.
__global__ void __launch_bounds__(CR_MAXWARPS * 32, 1)
    contract_fp64r_kernel(int N, int nu, int nd, int G, long long pairs, const double* __restrict__ Rc,
                          const double2* __restrict__ Theta, double2* __restrict__ vpair, double2* __restrict__ epair) {
    extern __shared__ double smr[];
    const int nt = nu + nd, Nnu = N * nu, nu2 = nu * nu, S2 = nu2 + nd * nd;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t per = contract_fp64r_warp_bytes(N, nu, nd) / sizeof(double);
    double2* sTh = reinterpret_cast<double2*>(smr + (size_t)warp * per);   // N x nt
    double* sR = reinterpret_cast<double*>(sTh + (size_t)N * nt);          // N x nu
    double2* sM = reinterpret_cast<double2*>(sR + ((size_t)Nnu + 1) / 2 * 2);   // S2
    const long long pair = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (pair >= pairs) return;
    const double2* gTh = Theta + pair * (long long)N * nt;
    for (int e = lane; e < N * nt; e += 32) sTh[e] = gTh[e];
    const double* Rp = Rc + pair * (long long)(G + 1) * Nnu;
    double2 eacc = cmk(0.0, 0.0);   // lane 0: one-body term + 1/2 sum_g v_g^2
    double2 exs = cmk(0.0, 0.0);    // this lane's share of sum_g Tr M_g^2 (reduced once, at the end)
    for (int g1 = 0; g1 <= G; ++g1) {
        const double* Rg = Rp + (long long)g1 * Nnu;
        __syncwarp();   // the previous matrix's reads of sR and sM are done
        for (int e = lane; e < Nnu; e += 32) sR[e] = Rg[e];
        __syncwarp();
        for (int e = lane; e < S2; e += 32) {
            int a, b, off;
            if (e < nu2) { a = e / nu; b = e - a * nu; off = 0; }
            else { const int q = e - nu2; a = q / nd; b = q - a * nd; off = nu; }
            const double* Ra = sR + a;
            const double2* Tb = sTh + off + b;
            double2 acc = cmk(0.0, 0.0);
            for (int k = 0; k < N; ++k) {
                const double r = Ra[(size_t)k * nu];
                const double2 t = Tb[(size_t)k * nt];
                acc.x = fma(r, t.x, acc.x);
                acc.y = fma(r, t.y, acc.y);
            }
            sM[e] = acc;
        }
        __syncwarp();
        double2 tr = cmk(0.0, 0.0);
        for (int e = lane; e < S2; e += 32) {
            int a, b, t;
            if (e < nu2) { a = e / nu; b = e - a * nu; t = b * nu + a; }
            else { const int q = e - nu2; a = q / nd; b = q - a * nd; t = nu2 + b * nd + a; }
            const double2 m = sM[e];
            if (g1 > 0) cfma(exs, m, sM[t]);
            if (a == b) tr = cadd(tr, m);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            tr.x += __shfl_xor_sync(0xffffffffu, tr.x, off);
            tr.y += __shfl_xor_sync(0xffffffffu, tr.y, off);
        }
        if (lane == 0) {
            if (g1 == 0) {
                eacc = cadd(eacc, tr);                   // one-body term sum_s Tr(Phi_s^T h Theta_s)
            } else {
                vpair[pair * G + (g1 - 1)] = tr;
                const double2 v2 = cmul(tr, tr);
                eacc.x += 0.5 * v2.x;
                eacc.y += 0.5 * v2.y;
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        exs.x += __shfl_xor_sync(0xffffffffu, exs.x, off);
        exs.y += __shfl_xor_sync(0xffffffffu, exs.y, off);
    }
    if (lane == 0) epair[pair] = cmk(eacc.x - 0.5 * exs.x, eacc.y - 0.5 * exs.y);
}

// Running count of refreshed pairs (counters[8]).
__global__ void rcache_count_kernel(const int* count, unsigned long long* counters) {
    counters[8] += (unsigned long long)*count;
}

cudaError_t rcache_refresh(cudaStream_t s, const Dims& d, const double* X, const double* Phi, int* dirty, int* list,
                           int* count, double* Rc, unsigned long long* counters) {
    if (d.pairs <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    rcache_collect_kernel<<<(unsigned)((d.pairs + 255) / 256), 256, 0, s>>>(d.pairs, dirty, list, count);
    const size_t smem = rcache_fill_smem(d.N, d.nu);
    if ((e = raise_smem_limit((const void*)rcache_fill_kernel, smem)) != cudaSuccess) return e;
    rcache_fill_kernel<<<4 * 152, RC_T, smem, s>>>(d.N, d.nu, d.G, X, Phi, list, count, Rc);
    rcache_count_kernel<<<1, 1, 0, s>>>(count, counters);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t contract_fp64r(cudaStream_t s, const Dims& d, const double* Rc, const double2* Theta, double2* vpair,
                           double2* epair) {
    if (!contract_fp64r_supported(d.N, d.nu, d.nd)) return cudaErrorInvalidValue;
    if (d.pairs <= 0) return cudaSuccess;
    const int warps = contract_fp64r_warps(d.N, d.nu, d.nd);
    const size_t smem = (size_t)warps * contract_fp64r_warp_bytes(d.N, d.nu, d.nd);
    cudaError_t e = raise_smem_limit((const void*)contract_fp64r_kernel, smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (d.pairs + warps - 1) / warps;
    contract_fp64r_kernel<<<(unsigned)blocks, warps * 32, smem, s>>>(d.N, d.nu, d.nd, d.G, d.pairs, Rc, Theta, vpair,
                                                                     epair);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace afq
