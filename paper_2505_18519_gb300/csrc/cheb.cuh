// Pieces shared by the Chebyshev kernels for Phi(x) = exp(S) Phi0 (Eq. (20)-(21)):
// block reductions, the expansion's coefficients, and the spectral interval.
//
// The series is exp(c + rho t) = e^c [I_0(rho) + 2 sum_k I_k(rho) T_k(t)] on an
// interval [c - rho, c + rho] holding the spectrum of the symmetric S.  The
// interval comes from a short Lanczos run on S in FP32 (the Gershgorin disks of
// the Lanczos tridiagonal, which includes the last residual, widened by 2 %,
// intersected with those of S): near the spectral interval, where the Gershgorin
// one of a sampled S is 3 to 4 times wider and would cost terms and cancellation.
// It is an estimate, not a bound, so the kernels check that the Chebyshev vectors
// do not grow and otherwise redo the problem on the Gershgorin interval.
#pragma once
#include <math.h>

#include "common.cuh"

namespace afq {

constexpr int CHEB_DF_MAX = 320;   // most terms of a series
constexpr int LZ_STEPS = 12;       // Lanczos steps of the spectral estimate
constexpr int LZ_NMAX = 256;       // largest N of the Lanczos vectors

// Sum over the block (up to 512 threads, a multiple of 32; red holds one value
// per warp); every thread gets the result, summed in warp order.
__device__ __forceinline__ float block_sum_f(float v, float* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();   // red may still be read from the previous call
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) t += red[w];
    return t;
}

// Chebyshev coefficients of exp on [c - rho, c + rho] (Miller's backward
// recurrence for I_k(rho), normalised by sum = e^rho), scaled by e^(c + rho);
// truncated at the first k with I_k(rho) < tol e^rho; returns the number of
// terms m.  One thread.
static __device__ int cheb_coefs(double c, double rho, double tol, double* coef, int* status) {
    int start = (int)ceil(rho) + 48;
    if (!isfinite(rho) || start > CHEB_DF_MAX) {
        atomicOr(status, STATUS_NONFINITE);
        start = CHEB_DF_MAX;
    }
    const double r2 = 2.0 / rho;
    double ip1 = 0.0, ik = 1e-280;
    for (int k = start; k >= 1; --k) {
        coef[k] = ik;
        const double im1 = fma((double)k * r2, ik, ip1);
        ip1 = ik;
        ik = im1;
        if (ik > 1e250) {   // rescale everything computed so far
            for (int j = k; j <= start; ++j) coef[j] *= 1e-250;
            ip1 *= 1e-250;
            ik *= 1e-250;
        }
    }
    coef[0] = ik;
    double norm = coef[0];
    for (int k = 1; k <= start; ++k) norm += 2.0 * coef[k];   // = e^rho in Miller's units
    int m = start;
    for (int k = 1; k <= start; ++k) {
        if (coef[k] < tol * norm) { m = k; break; }
    }
    const double scale = exp(c + rho) / norm;
    coef[0] *= scale;
    for (int k = 1; k <= m; ++k) coef[k] *= 2.0 * scale;
    return m;
}

// Shared-memory scratch of cheb_interval and its results.
struct ChebScratch {
    float red_lo[512], red_hi[512], red8[16];
    float lz_v[3][LZ_NMAX], lz_a[LZ_STEPS], lz_b[LZ_STEPS];
    double gers_c, gers_rho;   // Gershgorin interval of S (a bound)
    double est_c, est_rho;     // Lanczos estimate
};

// Both intervals of the symmetric N x N matrix S held in shared memory as FP32
// values S32[(i N + j) stride] (stride 2 reads the high parts of double-float
// pairs).  256 or 512 threads; ends with a barrier, after which every thread
// may read the results in sc.
__device__ __forceinline__ void cheb_interval(int N, const float* S32, int stride, ChebScratch& sc) {
    const int tid = threadIdx.x, nth = blockDim.x;
    // S is symmetric: row i is read as column i, so that the threads of a warp
    // (consecutive i) read consecutive words
    float lo = INFINITY, hi = -INFINITY;
    for (int i = tid; i < N; i += nth) {
        float r = 0.f;
        const float dgi = S32[((size_t)i * N + i) * stride];
        for (int j = 0; j < N; ++j)
            if (j != i) r += fabsf(S32[((size_t)j * N + i) * stride]);
        const float slack = 1e-5f * (r + fabsf(dgi)) + 1e-30f;   // keeps the FP32 sums a bound
        lo = fminf(lo, dgi - r - slack);
        hi = fmaxf(hi, dgi + r + slack);
    }
    sc.red_lo[tid] = lo;
    sc.red_hi[tid] = hi;
    __syncthreads();
    for (int off = nth / 2; off > 0; off >>= 1) {
        if (tid < off) {
            sc.red_lo[tid] = fminf(sc.red_lo[tid], sc.red_lo[tid + off]);
            sc.red_hi[tid] = fmaxf(sc.red_hi[tid], sc.red_hi[tid + off]);
        }
        __syncthreads();
    }
    const float g_lo = sc.red_lo[0], g_hi = sc.red_hi[0];
    // Lanczos on S from a fixed start vector
    for (int i = tid; i < N; i += nth) {
        sc.lz_v[0][i] = 0.f;
        sc.lz_v[1][i] = 1.f + 0.5f * __sinf(1.3f * (float)i + 0.7f);
    }
    float nrm = 0.f;
    for (int i = tid; i < N; i += nth) nrm += sc.lz_v[1][i] * sc.lz_v[1][i];
    nrm = block_sum_f(nrm, sc.red8);
    for (int i = tid; i < N; i += nth) sc.lz_v[1][i] *= rsqrtf(nrm);
    int ksteps = 0;
    float beta_prev = 0.f;
    // S v: `parts` threads per row when the rows fit the block (partial sums over every
    // parts-th column, added in a fixed order), else one thread per row
    const int Np = (N + 31) & ~31;
    const int parts = N <= nth ? nth / Np : 1;
    for (int j = 0; j < LZ_STEPS && j < N; ++j) {
        __syncthreads();
        float part = 0.f;
        if (parts > 1) {
            const int i = tid % Np, pr = tid / Np;
            float ps = 0.f;
            if (pr < parts && i < N)
                for (int q = pr; q < N; q += parts) ps = fmaf(S32[((size_t)q * N + i) * stride], sc.lz_v[1][q], ps);
            if (pr < parts) sc.red_lo[pr * Np + i] = ps;
            __syncthreads();
            if (tid < N) {
                float wsum = 0.f;
                for (int r = 0; r < parts; ++r) wsum += sc.red_lo[r * Np + tid];
                sc.lz_v[2][tid] = wsum;
                part = wsum * sc.lz_v[1][tid];
            }
        } else {
            for (int i = tid; i < N; i += nth) {
                float wsum = 0.f;
                for (int q = 0; q < N; ++q) wsum = fmaf(S32[((size_t)q * N + i) * stride], sc.lz_v[1][q], wsum);
                sc.lz_v[2][i] = wsum;
                part = fmaf(wsum, sc.lz_v[1][i], part);
            }
        }
        const float alpha = block_sum_f(part, sc.red8);
        float part2 = 0.f;
        for (int i = tid; i < N; i += nth) {
            const float wv = sc.lz_v[2][i] - alpha * sc.lz_v[1][i] - beta_prev * sc.lz_v[0][i];
            sc.lz_v[2][i] = wv;
            part2 = fmaf(wv, wv, part2);
        }
        const float beta = sqrtf(block_sum_f(part2, sc.red8));
        if (tid == 0) { sc.lz_a[j] = alpha; sc.lz_b[j] = beta; }
        ksteps = j + 1;
        if (!(beta > 1e-6f * (fabsf(alpha) + 1e-30f))) break;   // invariant subspace found
        const float ib = 1.f / beta;
        for (int i = tid; i < N; i += nth) {
            sc.lz_v[0][i] = sc.lz_v[1][i];
            sc.lz_v[1][i] = sc.lz_v[2][i] * ib;
        }
        beta_prev = beta;
    }
    __syncthreads();
    if (tid == 0) {
        float tl = INFINITY, th = -INFINITY;
        for (int j = 0; j < ksteps; ++j) {
            const float r = (j > 0 ? fabsf(sc.lz_b[j - 1]) : 0.f) + fabsf(sc.lz_b[j]);
            tl = fminf(tl, sc.lz_a[j] - r);
            th = fmaxf(th, sc.lz_a[j] + r);
        }
        const float margin = 0.02f * (th - tl) + 1e-6f;
        const double elo = fmax((double)g_lo, (double)(tl - margin)), ehi = fmin((double)g_hi, (double)(th + margin));
        sc.gers_c = 0.5 * ((double)g_lo + (double)g_hi);
        sc.gers_rho = fmax(0.5 * ((double)g_hi - (double)g_lo), 1e-3);
        if (ehi > elo && isfinite(elo) && isfinite(ehi)) {
            sc.est_c = 0.5 * (elo + ehi);
            sc.est_rho = fmax(0.5 * (ehi - elo), 1e-3);
        } else {
            sc.est_c = sc.gers_c;
            sc.est_rho = sc.gers_rho;
        }
    }
    __syncthreads();
}

}  // namespace afq
