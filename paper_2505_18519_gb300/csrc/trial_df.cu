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
// The series is the Chebyshev expansion exp(c + rho t) = e^c [I_0(rho) +
// 2 sum_k I_k(rho) T_k(t)] on an interval [c - rho, c + rho] holding the
// spectrum of S, modified Bessel I_k by Miller's backward recurrence in FP64
// (one thread, scalar), truncated once the coefficients fall below 1e-18 of
// e^rho (1e-15 when the recurrence runs in double-float, about 2^-44).  The partial sums cancel by about e^(rho - rho_true) when rho
// overestimates the spectral half-width, which multiplies the rounding error
// and the number of terms; the Gershgorin half-width of the sampled S is
// 3 to 4 times the spectral one.  So the interval comes from a short Lanczos
// run, checked a posteriori (see chebyshev_expm_df_kernel).
#include <algorithm>

#include "cheb.cuh"
#include "df.cuh"
#include "kernels.cuh"

namespace afq {

constexpr double RHO_DF = 6.5;   // largest Gershgorin half-width run in double-float

// Interval of the expansion: first an estimate from LZ_STEPS Lanczos steps on S
// (FP32; the Gershgorin disks of the Lanczos tridiagonal, which includes the
// last residual, widened by 2 %, intersected with those of S), which is near
// the spectral interval where the Gershgorin one of S can be several times
// wider.  Estimates are not bounds, so the recurrence checks that the
// Chebyshev vectors do not grow (|T_k(t)| <= 1 on the spectrum keeps
// ||V_k||_F <= ||Phi0||_F); if they do, the problem is done again on the
// Gershgorin interval of S, in double-float if its half-width is at most
// RHO_DF and in FP64 otherwise.
// One problem per call; the whole block of 256 threads takes part.  s_global (with
// s_is_df): S stays in global memory and is read from there (L2) by every term, for
// N too large for S in shared memory; shared memory then holds the vectors only.
__device__ __forceinline__ void cheb_df_problem(long long prob, int N, int nu, const double* __restrict__ S_all,
                                                const double* __restrict__ Phi0, double* __restrict__ Out,
                                                const int* __restrict__ alive, int P, int* status, int allow_df,
                                                int s_is_df, int s_global = 0) {
    extern __shared__ dfl smf[];
    __shared__ double coef[CHEB_DF_MAX + 2];
    __shared__ dfl coefd[CHEB_DF_MAX + 2];
    __shared__ ChebScratch sc;
    float* red8 = sc.red8;
    __shared__ int nterms, mode;
    __shared__ dfl cshift_d, irho_d;
    __shared__ double cshift, irho;
    if (alive && !alive[prob / P]) return;
    const double* Sg = S_all + prob * (long long)N * N;
    const dfl* Sgd = reinterpret_cast<const dfl*>(Sg);
    dfl* Ssm = smf;
    const dfl* S = s_global ? Sgd : Ssm;
    dfl* Vp = smf + (s_global ? (size_t)0 : (size_t)N * N);
    dfl* Vc = Vp + (size_t)N * nu;
    dfl* acc = Vc + (size_t)N * nu;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int nn = N * nu;
    // S to double-float (or as given, when the caller formed it in double-float);
    // the Gershgorin interval and the Lanczos estimate from its high parts
    if (!s_global)
        for (int e = tid; e < N * N; e += nth) Ssm[e] = s_is_df ? Sgd[e] : df_from(Sg[e]);
    __syncthreads();
    cheb_interval(N, &S[0].hi, 2, sc);
    float phi_ss = 0.f;   // ||Phi0||_F^2
    for (int e = tid; e < nn; e += nth) phi_ss = fmaf((float)Phi0[e], (float)Phi0[e], phi_ss);
    phi_ss = block_sum_f(phi_ss, red8);
    const float grow_limit = 1.5625f * phi_ss + 1e-30f;   // ||V_k||_F <= 1.25 ||Phi0||_F

    for (int attempt = 0; attempt < 2; ++attempt) {
        if (tid == 0) {
            const double c = attempt == 0 ? sc.est_c : sc.gers_c, rho = attempt == 0 ? sc.est_rho : sc.gers_rho;
            // 0 double-float with the growth check, 1 double-float, 2 FP64 with the
            // growth check, 3 FP64
            if (allow_df) mode = attempt == 0 ? 0 : (rho <= RHO_DF ? 1 : 3);
            else mode = attempt == 0 ? 2 : 3;
            // truncation below the arithmetic's own resolution: about 2^-44 in double-float
            // (1e-15 of e^rho), FP64 rounding (1e-18)
            const int m = cheb_coefs(c, rho, mode < 2 ? 1e-15 : 1e-18, coef, status);
            for (int k = 0; k <= m; ++k) coefd[k] = df_from(coef[k]);
            nterms = m;
            cshift = c;
            irho = 1.0 / rho;
            cshift_d = df_from(c);
            irho_d = df_from(1.0 / rho);
        }
        __syncthreads();
        const int m = nterms;
        if (mode >= 2) {
            // FP64 recurrence; S, V and the sum in FP64 (8 bytes per element, same storage)
            const bool check64 = mode == 2;
            double* S64 = reinterpret_cast<double*>(smf);
            double* Vp64 = reinterpret_cast<double*>(Vp);
            double* Vc64 = reinterpret_cast<double*>(Vc);
            double* acc64 = reinterpret_cast<double*>(acc);
            if (!s_global)
                for (int e = tid; e < N * N; e += nth) S64[e] = s_is_df ? df_to(Sgd[e]) : Sg[e];
            __syncthreads();
            const double c = cshift, ir = irho;
            for (int e = tid; e < nn; e += nth) {
                Vp64[e] = Phi0[e];
                acc64[e] = coef[0] * Phi0[e];
            }
            __syncthreads();
            bool grew64 = false;
            for (int k = 1; k <= m && !grew64; ++k) {
                const double* Vsrc = k == 1 ? Vp64 : Vc64;
                float ss64 = 0.f;
                for (int e = tid; e < nn; e += nth) {
                    const int i = e / nu, a = e - i * nu;
                    double sum = 0.0;
                    if (s_global)   // S as double-float pairs in global memory, rounded to FP64 per use
                        for (int j = 0; j < N; ++j) sum = fma(df_to(Sgd[(size_t)i * N + j]), Vsrc[j * nu + a], sum);
                    else
                        for (int j = 0; j < N; ++j) sum = fma(S64[(size_t)i * N + j], Vsrc[j * nu + a], sum);
                    sum = (sum - c * Vsrc[e]) * ir;
                    double v;
                    if (k == 1) {
                        v = sum;
                        Vc64[e] = v;
                    } else {
                        v = 2.0 * sum - Vp64[e];
                        Vp64[e] = v;
                    }
                    acc64[e] = fma(coef[k], v, acc64[e]);
                    if (check64) {
                        const float vf = __double2float_rn(v);
                        ss64 = fmaf(vf, vf, ss64);
                    }
                }
                if (check64) grew64 = block_sum_f(ss64, red8) > grow_limit;   // uniform across the block
                else __syncthreads();
                if (k >= 2) { double* t = Vp64; Vp64 = Vc64; Vc64 = t; }
            }
            if (grew64) {       // the estimate missed part of the spectrum: start again
                __syncthreads();
                continue;
            }
            __syncthreads();
            double* o = Out + prob * (long long)nn;
            for (int e = tid; e < nn; e += nth) o[e] = acc64[e];
            return;
        }
        const dfl cs = cshift_d, ir = irho_d;
        const bool check = mode == 0;
        // t V for one element: ((S V)_e - c V_e) / rho, the product by Dot2
        auto tv = [&](const dfl* V, int e) -> dfl {
            const int i = e / nu, a = e - i * nu;
            const dfl* Srow = S + (size_t)i * N;
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
        // the same for elements e0 and e0 + 1 of one row (n_up even, e0 even): one load
        // of S per term serves both, each element's Dot2 sequence is unchanged
        auto tv2 = [&](const dfl* V, int e0, dfl& r0, dfl& r1) {
            const int i = e0 / nu, a = e0 - i * nu;
            const dfl* Srow = S + (size_t)i * N;
            const dfl* Va = V + a;
            float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
            for (int j = 0; j < N; ++j) {
                const dfl x = Srow[j], y0 = Va[(size_t)j * nu], y1 = Va[(size_t)j * nu + 1];
                dot2_fma(s0, c0, x, y0);
                dot2_fma(s1, c1, x, y1);
            }
            r0 = df_mul(df_add(df_two_sum(s0, c0), df_neg(df_mul(cs, V[e0]))), ir);
            r1 = df_mul(df_add(df_two_sum(s1, c1), df_neg(df_mul(cs, V[e0 + 1]))), ir);
        };
        const bool pairs2 = (nu & 1) == 0;
        for (int e = tid; e < nn; e += nth) {
            const dfl f = df_from(Phi0[e]);
            Vp[e] = f;
            acc[e] = df_mul(coefd[0], f);
        }
        __syncthreads();
        float ss = 0.f;
        if (pairs2) {
            for (int e = 2 * tid; e < nn; e += 2 * nth) {
                dfl sv[2];
                tv2(Vp, e, sv[0], sv[1]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    Vc[e + h] = sv[h];
                    acc[e + h] = df_add(acc[e + h], df_mul(coefd[1], sv[h]));
                    ss = fmaf(sv[h].hi, sv[h].hi, ss);
                }
            }
        } else {
            for (int e = tid; e < nn; e += nth) {
                const dfl sv = tv(Vp, e);
                Vc[e] = sv;
                acc[e] = df_add(acc[e], df_mul(coefd[1], sv));
                ss = fmaf(sv.hi, sv.hi, ss);
            }
        }
        bool grew = check && block_sum_f(ss, red8) > grow_limit;
        for (int k = 2; k <= m && !grew; ++k) {
            // V_k = 2 t V_{k-1} - V_{k-2}, written over V_{k-2} element by element
            __syncthreads();
            ss = 0.f;
            if (pairs2) {
                for (int e = 2 * tid; e < nn; e += 2 * nth) {
                    dfl sv[2];
                    tv2(Vc, e, sv[0], sv[1]);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const dfl v = df_add(dfl{2.f * sv[h].hi, 2.f * sv[h].lo}, df_neg(Vp[e + h]));
                        Vp[e + h] = v;
                        acc[e + h] = df_add(acc[e + h], df_mul(coefd[k], v));
                        ss = fmaf(v.hi, v.hi, ss);
                    }
                }
            } else {
                for (int e = tid; e < nn; e += nth) {
                    const dfl sv = tv(Vc, e);
                    const dfl v = df_add(dfl{2.f * sv.hi, 2.f * sv.lo}, df_neg(Vp[e]));
                    Vp[e] = v;
                    acc[e] = df_add(acc[e], df_mul(coefd[k], v));
                    ss = fmaf(v.hi, v.hi, ss);
                }
            }
            if (check) grew = block_sum_f(ss, red8) > grow_limit;   // uniform across the block
            else __syncthreads();
            dfl* t = Vp; Vp = Vc; Vc = t;
        }
        if (grew) {           // the estimate missed part of the spectrum: start again
            __syncthreads();
            continue;
        }
        __syncthreads();
        double* o = Out + prob * (long long)nn;
        for (int e = tid; e < nn; e += nth) o[e] = df_to(acc[e]);
        return;
    }
}

__global__ void __launch_bounds__(256) chebyshev_expm_df_kernel(int N, int nu, const double* __restrict__ S_all,
                                                                const double* __restrict__ Phi0, double* __restrict__ Out,
                                                                const int* __restrict__ alive, int P, int* status,
                                                                int allow_df, int s_is_df, int s_global) {
    cheb_df_problem(blockIdx.x, N, nu, S_all, Phi0, Out, alive, P, status, allow_df, s_is_df, s_global);
}

// The problems list[0 .. *count), grid-stride (the tensor-core kernel's redo list).
__global__ void __launch_bounds__(256) chebyshev_expm_df_list_kernel(int N, int nu, const double* __restrict__ S_all,
                                                                     const double* __restrict__ Phi0,
                                                                     double* __restrict__ Out,
                                                                     const int* __restrict__ alive, int P, int* status,
                                                                     int s_is_df, const int* __restrict__ list,
                                                                     const int* __restrict__ count) {
    const int n = *count;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        cheb_df_problem(list[i], N, nu, S_all, Phi0, Out, alive, P, status, 1, s_is_df);
        __syncthreads();   // the shared memory is reused by the next problem
    }
}

// Same contract as trial_orbitals (S_all is only read).
bool trial_orbitals_df_supported(int N, int nu) {
    return (3 * (size_t)N * nu + (size_t)N * N) * sizeof(dfl) <= 200 * 1024 && N <= LZ_NMAX;
}

// The double-float kernel with S read from global memory (double-float S).
bool trial_orbitals_dfg_supported(int N, int nu) {
    return 3 * (size_t)N * nu * sizeof(dfl) <= 200 * 1024 && N <= LZ_NMAX;
}

static cudaError_t trial_orbitals_lanczos(cudaStream_t s, int N, int nu, long long problems, double* S_all,
                                          const double* Phi0, double* Out, const int* alive, int P, int* status,
                                          int threads, bool allow_df, bool s_is_df) {
    if (problems <= 0) return cudaSuccess;
    // S in shared memory, or (double-float S that does not fit there) read from global memory
    const bool s_global = !trial_orbitals_df_supported(N, nu) && s_is_df && trial_orbitals_dfg_supported(N, nu);
    const size_t bytes = (3 * (size_t)N * nu + (s_global ? (size_t)0 : (size_t)N * N)) * sizeof(dfl);
    if (!trial_orbitals_df_supported(N, nu) && !s_global) {   // the Gershgorin FP64 kernel
        if (s_is_df) return cudaErrorInvalidValue;
        return trial_orbitals_gershgorin(s, N, nu, problems, S_all, Phi0, Out, alive, P, status, threads);
    }
    cudaError_t e = raise_smem_limit((const void*)chebyshev_expm_df_kernel, bytes);
    if (e != cudaSuccess) return e;
    chebyshev_expm_df_kernel<<<(unsigned)problems, 256, bytes, s>>>(N, nu, S_all, Phi0, Out, alive, P, status,
                                                                   allow_df ? 1 : 0, s_is_df ? 1 : 0, s_global ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t trial_orbitals_df(cudaStream_t s, int N, int nu, long long problems, double* S_all, const double* Phi0,
                              double* Out, const int* alive, int P, int* status, int threads, bool s_is_df) {
    return trial_orbitals_lanczos(s, N, nu, problems, S_all, Phi0, Out, alive, P, status, threads, true, s_is_df);
}

cudaError_t trial_orbitals_df_list(cudaStream_t s, int N, int nu, const double* S_all, bool s_is_df, const double* Phi0,
                                   double* Out, const int* alive, int P, int* status, const int* list,
                                   const int* count) {
    if (!trial_orbitals_df_supported(N, nu)) return cudaErrorInvalidValue;
    const size_t bytes = (3 * (size_t)N * nu + (size_t)N * N) * sizeof(dfl);
    cudaError_t e = raise_smem_limit((const void*)chebyshev_expm_df_list_kernel, bytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    chebyshev_expm_df_list_kernel<<<(unsigned)std::max(1, sms), 256, bytes, s>>>(N, nu, S_all, Phi0, Out, alive, P,
                                                                                 status, s_is_df ? 1 : 0, list, count);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t trial_orbitals(cudaStream_t s, int N, int nu, long long problems, const double* S_all, const double* Phi0,
                           double* Out, const int* alive, int P, int* status, int threads) {
    return trial_orbitals_lanczos(s, N, nu, problems, const_cast<double*>(S_all), Phi0, Out, alive, P, status, threads,
                                  false, false);
}

// ---------------------------------------------------------------- S = X U in double-float
// S[p, e] = sum_k X[p, k] U[k, e] for the proposal matrices S_p = sum_k x'_k U_k
// (the mixed-precision path): X (M x K, FP64) is rounded to double-float as its
// tiles are loaded, U comes in double-float from init, each product is
// accumulated by Dot2, and S is stored as double-float pairs (8 bytes per
// element, the layout chebyshev_expm_df_kernel reads with s_is_df).
constexpr int DG_T = 64, DG_K = 16;

__global__ void u_to_df_kernel(long long n, const double* __restrict__ U, dfl* __restrict__ Ud) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        Ud[e] = df_from(U[e]);
}

// XDF: X already in double-float (Xd); else rounded from FP64 as its tiles load.
template <bool XDF>
__global__ void __launch_bounds__(256) gemm_df_kernel(int M, int Nc, int K, const double* __restrict__ X,
                                                      const dfl* __restrict__ Xd, const dfl* __restrict__ Ud,
                                                      dfl* __restrict__ S) {
    __shared__ dfl Xs[DG_K][DG_T + 1];
    __shared__ dfl Us[DG_K][DG_T];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const long long row0 = (long long)blockIdx.y * DG_T, col0 = (long long)blockIdx.x * DG_T;
    float sh[4][4], sl[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { sh[i][j] = 0.f; sl[i][j] = 0.f; }
    for (int k0 = 0; k0 < K; k0 += DG_K) {
        for (int e = threadIdx.x; e < DG_K * DG_T; e += 256) {
            const int r = e / DG_K, kk = e % DG_K;        // X tile: 64 rows x 16 k
            const long long gr = row0 + r;
            const int gk = k0 + kk;
            if constexpr (XDF) Xs[kk][r] = (gr < M && gk < K) ? Xd[gr * K + gk] : dfl{0.f, 0.f};
            else Xs[kk][r] = (gr < M && gk < K) ? df_from(X[gr * K + gk]) : dfl{0.f, 0.f};
            const int kb = e / DG_T, c = e % DG_T;        // U tile: 16 k x 64 cols
            const long long gc = col0 + c;
            const int gkb = k0 + kb;
            Us[kb][c] = (gkb < K && gc < Nc) ? Ud[(long long)gkb * Nc + gc] : dfl{0.f, 0.f};
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < DG_K; ++kk) {
            dfl a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Xs[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Us[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float p = a[i].hi * b[j].hi;
                    float q = fmaf(a[i].hi, b[j].hi, -p);
                    q = fmaf(a[i].hi, b[j].lo, q);
                    q = fmaf(a[i].lo, b[j].hi, q);
                    const float t = sh[i][j] + p, z = t - sh[i][j];
                    sl[i][j] += q + ((sh[i][j] - (t - z)) + (p - z));
                    sh[i][j] = t;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long r = row0 + ty + 16 * i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long c = col0 + tx + 16 * j;
            if (c < Nc) S[r * Nc + c] = df_two_sum(sh[i][j], sl[i][j]);
        }
    }
}

cudaError_t u_to_df(cudaStream_t s, long long n, const double* U, void* Ud) {
    if (n <= 0) return cudaSuccess;
    u_to_df_kernel<<<(unsigned)min((n + 255) / 256, 4096LL), 256, 0, s>>>(n, U, reinterpret_cast<dfl*>(Ud));
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t gemm_df(cudaStream_t s, int M, int Nc, int K, const double* X, const void* Ud, double* S, void* Xdf) {
    if (M <= 0 || Nc <= 0) return cudaSuccess;
    dim3 grid((unsigned)((Nc + DG_T - 1) / DG_T), (unsigned)((M + DG_T - 1) / DG_T));
    if (Xdf) {   // X to double-float once (its FP64 rounding would otherwise run once per column tile)
        const cudaError_t e = u_to_df(s, (long long)M * K, X, Xdf);
        if (e != cudaSuccess) return e;
        gemm_df_kernel<true><<<grid, 256, 0, s>>>(M, Nc, K, X, reinterpret_cast<const dfl*>(Xdf),
                                                  reinterpret_cast<const dfl*>(Ud), reinterpret_cast<dfl*>(S));
    } else {
        gemm_df_kernel<false><<<grid, 256, 0, s>>>(M, Nc, K, X, nullptr, reinterpret_cast<const dfl*>(Ud),
                                                   reinterpret_cast<dfl*>(S));
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace afq
