// Trial orbitals Phi(x) = exp(S) Phi0 (Eq. (20)-(21), one symmetric
// S = sum_k x_k U_k per path) for the mixed-precision path, in double-float
// arithmetic: every value is an unevaluated sum hi + lo of two FP32 numbers,
// products and sums use error-free transformations (TwoProduct by fmaf,
// Knuth's TwoSum), and the dot products of the matrix-vector products follow
// the compensated Dot2 scheme of Ogita, Rump and Oishi (2005) with the
// cross terms of the low parts.  That gives about 44 significant bits, far
// more than the split-FP16 contraction of the same path needs, at FP32
// instruction rates: FP64 arithmetic is about 64 times slower than FP32 on
// this part, and the FP64 version of this kernel is FP64-pipe bound.
//
// The series is the same Chebyshev expansion as the FP64 kernel: exp(c + rho t)
// = e^c [I_0(rho) + 2 sum_k I_k(rho) T_k(t)] on the Gershgorin interval
// [c - rho, c + rho] of S (bounds formed in FP32 and widened by a relative
// 1e-5 so they stay bounds), modified Bessel I_k by Miller's backward
// recurrence in FP64 (one thread, scalar), truncated once the coefficients
// fall below 1e-18 of e^rho.  The partial sums cancel by about e^(rho - rho_true)
// when the Gershgorin half-width rho overestimates the spectral one, which
// multiplies the rounding error; a problem whose rho exceeds RHO_DF (the
// large workload's S have rho ~ 13) runs the same recurrence in FP64 instead,
// so the result stays within ~1e-9 relative of exp(S) Phi0 either way.
#include "kernels.cuh"

namespace afq {

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl df_quick(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    const dfl s = df_two_sum(a.hi, b.hi), t = df_two_sum(a.lo, b.lo);
    const dfl u = df_quick(s.hi, s.lo + t.hi);
    return df_quick(u.hi, u.lo + t.lo);
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_quick(p, e);
}
__device__ __forceinline__ dfl df_from(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }

constexpr int CHEB_DF_MAX = 320;
constexpr double RHO_DF = 6.5;   // largest Gershgorin half-width run in double-float

template <bool S_SMEM>
__global__ void __launch_bounds__(256) chebyshev_expm_df_kernel(int N, int nu, long long problems,
                                                                const double* __restrict__ S_all,
                                                                const double* __restrict__ Phi0, double* __restrict__ Out,
                                                                const int* __restrict__ alive, int P, int* status) {
    extern __shared__ dfl smf[];
    __shared__ double coef[CHEB_DF_MAX + 2];
    __shared__ dfl coefd[CHEB_DF_MAX + 2];
    __shared__ float red_lo[256], red_hi[256];
    __shared__ int nterms, use_df;
    __shared__ dfl cshift_d, irho_d;
    __shared__ double cshift, irho;
    const long long prob = blockIdx.x;
    if (alive && !alive[prob / P]) return;
    const double* Sg = S_all + prob * (long long)N * N;
    dfl* S = S_SMEM ? smf : nullptr;
    dfl* Vp = S_SMEM ? smf + (size_t)N * N : smf;
    dfl* Vc = Vp + (size_t)N * nu;
    dfl* acc = Vc + (size_t)N * nu;
    dfl* Sd = reinterpret_cast<dfl*>(const_cast<double*>(Sg));   // in place when S is not in shared memory
    const int tid = threadIdx.x, nth = blockDim.x;
    // Gershgorin interval in FP32 (row sums of |S_ij|), S to double-float
    float lo = INFINITY, hi = -INFINITY;
    for (int i = tid; i < N; i += nth) {
        float r = 0.f, dgi = 0.f;
        for (int j = 0; j < N; ++j) {
            const double x = Sg[(long long)i * N + j];
            const float xf = __double2float_rn(x);
            if (j == i) dgi = xf;
            else r += fabsf(xf);
        }
        const float slack = 1e-5f * (r + fabsf(dgi)) + 1e-30f;
        lo = fminf(lo, dgi - r - slack);
        hi = fmaxf(hi, dgi + r + slack);
    }
    red_lo[tid] = lo;
    red_hi[tid] = hi;
    __syncthreads();
    for (int off = nth / 2; off > 0; off >>= 1) {
        if (tid < off) {
            red_lo[tid] = fminf(red_lo[tid], red_lo[tid + off]);
            red_hi[tid] = fmaxf(red_hi[tid], red_hi[tid + off]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        const double c = 0.5 * ((double)red_lo[0] + (double)red_hi[0]);
        const double rho = fmax(0.5 * ((double)red_hi[0] - (double)red_lo[0]), 1e-3);
        int start = (int)ceil(rho) + 48;
        if (!isfinite(rho) || start > CHEB_DF_MAX) {
            atomicOr(status, STATUS_NONFINITE);
            start = CHEB_DF_MAX;
        }
        // Miller: I_{k-1} = (2k / rho) I_k + I_{k+1}, started at order `start` with I = 0, 1.
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
            if (coef[k] < 1e-18 * norm) { m = k; break; }
        }
        const double scale = exp(c + rho) / norm;
        coef[0] *= scale;
        for (int k = 1; k <= m; ++k) coef[k] *= 2.0 * scale;
        for (int k = 0; k <= m; ++k) coefd[k] = df_from(coef[k]);
        nterms = m;
        cshift = c;
        irho = 1.0 / rho;
        cshift_d = df_from(c);
        irho_d = df_from(1.0 / rho);
        use_df = rho <= RHO_DF;
    }
    __syncthreads();
    const int m = nterms;
    const int nn = N * nu;
    if (!use_df) {
        // FP64 recurrence (same storage: 8 bytes per element)
        double* S64 = S_SMEM ? reinterpret_cast<double*>(smf) : nullptr;
        double* Vp64 = reinterpret_cast<double*>(Vp);
        double* Vc64 = reinterpret_cast<double*>(Vc);
        double* acc64 = reinterpret_cast<double*>(acc);
        if (S_SMEM)
            for (int e = tid; e < N * N; e += nth) S64[e] = Sg[e];
        __syncthreads();
        const double* Sr = S_SMEM ? S64 : Sg;
        const double c = cshift, ir = irho;
        for (int e = tid; e < nn; e += nth) {
            Vp64[e] = Phi0[e];
            acc64[e] = coef[0] * Phi0[e];
        }
        __syncthreads();
        for (int k = 1; k <= m; ++k) {
            const double* Vsrc = k == 1 ? Vp64 : Vc64;
            for (int e = tid; e < nn; e += nth) {
                const int i = e / nu, a = e - i * nu;
                double sum = 0.0;
                for (int j = 0; j < N; ++j) sum = fma(Sr[(long long)i * N + j], Vsrc[j * nu + a], sum);
                sum = (sum - c * Vsrc[e]) * ir;
                if (k == 1) {
                    Vc64[e] = sum;
                    acc64[e] = fma(coef[1], sum, acc64[e]);
                } else {
                    const double v = 2.0 * sum - Vp64[e];
                    Vp64[e] = v;
                    acc64[e] = fma(coef[k], v, acc64[e]);
                }
            }
            __syncthreads();
            if (k >= 2) { double* t = Vp64; Vp64 = Vc64; Vc64 = t; }
        }
        double* o = Out + prob * (long long)nn;
        for (int e = tid; e < nn; e += nth) o[e] = acc64[e];
        return;
    }
    if (S_SMEM) {
        for (int e = tid; e < N * N; e += nth) S[e] = df_from(Sg[e]);
    } else {
        // convert in place: each element is read and written by the same thread
        for (int e = tid; e < N * N; e += nth) Sd[e] = df_from(Sg[e]);
    }
    __syncthreads();
    const dfl* Sr = S_SMEM ? S : Sd;
    const dfl cs = cshift_d, ir = irho_d;
    // t V for one element: ((S V)_e - c V_e) / rho, the product by Dot2
    auto tv = [&](const dfl* V, int e) -> dfl {
        const int i = e / nu, a = e - i * nu;
        const dfl* Srow = Sr + (size_t)i * N;
        float s = 0.f, cc = 0.f;
        for (int j = 0; j < N; ++j) {
            const dfl x = Srow[j], y = V[(size_t)j * nu + a];
            const float p = x.hi * y.hi;
            float q = fmaf(x.hi, y.hi, -p);
            q = fmaf(x.hi, y.lo, q);
            q = fmaf(x.lo, y.hi, q);
            const float t = s + p, z = t - s;
            cc += q + ((s - (t - z)) + (p - z));
            s = t;
        }
        const dfl sv = df_two_sum(s, cc);
        return df_mul(df_add(sv, df_neg(df_mul(cs, V[e]))), ir);
    };
    for (int e = tid; e < nn; e += nth) {
        const dfl f = df_from(Phi0[e]);
        Vp[e] = f;
        acc[e] = df_mul(coefd[0], f);
    }
    __syncthreads();
    for (int e = tid; e < nn; e += nth) {
        const dfl s = tv(Vp, e);
        Vc[e] = s;
        acc[e] = df_add(acc[e], df_mul(coefd[1], s));
    }
    __syncthreads();
    for (int k = 2; k <= m; ++k) {
        // V_k = 2 t V_{k-1} - V_{k-2}, written over V_{k-2} element by element
        for (int e = tid; e < nn; e += nth) {
            const dfl s = tv(Vc, e);
            const dfl v = df_add(dfl{2.f * s.hi, 2.f * s.lo}, df_neg(Vp[e]));
            Vp[e] = v;
            acc[e] = df_add(acc[e], df_mul(coefd[k], v));
        }
        __syncthreads();
        dfl* t = Vp; Vp = Vc; Vc = t;
    }
    double* o = Out + prob * (long long)nn;
    for (int e = tid; e < nn; e += nth) o[e] = df_to(acc[e]);
}

// Same contract as trial_orbitals; S_all is overwritten (converted in place)
// when S does not fit in shared memory.
cudaError_t trial_orbitals_df(cudaStream_t s, int N, int nu, long long problems, double* S_all, const double* Phi0,
                              double* Out, const int* alive, int P, int* status, int threads) {
    if (problems <= 0) return cudaSuccess;
    if (threads != 128 && threads != 256) threads = 256;
    const size_t vec = 3 * (size_t)N * nu * sizeof(dfl);
    const size_t full = vec + (size_t)N * N * sizeof(dfl);
    cudaError_t e;
    if (full <= 200 * 1024) {
        e = raise_smem_limit((const void*)chebyshev_expm_df_kernel<true>, full);
        if (e != cudaSuccess) return e;
        chebyshev_expm_df_kernel<true><<<(unsigned)problems, threads, full, s>>>(N, nu, problems, S_all, Phi0, Out, alive, P,
                                                                                 status); count_launches(1);
    } else {
        if (vec > 200 * 1024) return cudaErrorInvalidValue;
        e = raise_smem_limit((const void*)chebyshev_expm_df_kernel<false>, vec);
        if (e != cudaSuccess) return e;
        chebyshev_expm_df_kernel<false><<<(unsigned)problems, threads, vec, s>>>(N, nu, problems, S_all, Phi0, Out, alive, P,
                                                                                 status); count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace afq
