// FP64 small-matrix kernels of the step: overlaps with batched LU, the
// Theta = phi (Phi^T phi)^-1 matrices, re-orthonormalisation, the trial
// orbitals Phi(x) = exp(S) Phi0 by a Chebyshev series, a plain FP64 GEMM, and the
// init-time one-body propagator exp(-tau T / 2).
#include "df.cuh"
#include "kernels.cuh"

namespace afq {

// ---------------------------------------------------------------- GEMM
// C[M x Nc] = alpha * A[M x K] * B[K x Nc] + beta * C, row-major with leading
// dimensions.  64 x 64 output tile per 256-thread block, 4 x 4 per thread.
__global__ void __launch_bounds__(256) gemm_nn_f64_kernel(int M, int Nc, int K, double alpha, const double* __restrict__ A,
                                                          long long lda, const double* __restrict__ B, long long ldb,
                                                          double beta, double* __restrict__ C, long long ldc) {
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64];
    int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    long long row0 = (long long)blockIdx.y * 64, col0 = (long long)blockIdx.x * 64;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            int r = e / 16, kk = e % 16;          // A tile: 64 rows x 16 k
            long long gr = row0 + r;
            int gk = k0 + kk;
            As[kk][r] = (gr < M && gk < K) ? A[gr * lda + gk] : 0.0;
            int kb = e / 64, c = e % 64;          // B tile: 16 k x 64 cols
            long long gc = col0 + c;
            int gkb = k0 + kb;
            Bs[kb][c] = (gkb < K && gc < Nc) ? B[(long long)gkb * ldb + gc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        long long r = row0 + ty + 16 * i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            long long c = col0 + tx + 16 * j;
            if (c >= Nc) continue;
            double v = alpha * acc[i][j];
            if (beta != 0.0) v = fma(beta, C[r * ldc + c], v);
            C[r * ldc + c] = v;
        }
    }
}

void gemm_nn_f64(cudaStream_t s, int M, int Nc, int K, double alpha, const double* A, long long lda, const double* B,
                 long long ldb, double beta, double* C, long long ldc) {
    if (M <= 0 || Nc <= 0) return;
    dim3 grid((unsigned)((Nc + 63) / 64), (unsigned)((M + 63) / 64));
    gemm_nn_f64_kernel<<<grid, 256, 0, s>>>(M, Nc, K, alpha, A, lda, B, ldb, beta, C, ldc); count_launches(1);
}

// ---------------------------------------------------------------- overlap + LU
// One warp per (pair, spin).  A = Phi_s^T phi_s (n x n complex; Phi real),
// LU with partial pivoting (largest |re|+|im|, lowest row on ties),
// log det A = sum log|u_kk| + i Arg(prod u_kk / |u_kk| * (-1)^swaps).
// With Theta != nullptr also A^-1 (from the LU) and, by `trial_side`:
//   OVL_THETA (0): Theta_s = phi_s A^-1 in columns col0..col0+n-1 of Theta[pair] (N x nt);
//   OVL_TRIAL (1): the trial-side factor B_s = Phi_s A^-T there instead (then
//                  Phi_s^T X Theta_s = A B_s^T X phi_s A^-1 has the same traces);
//   OVL_INVERSE (2): A^-1 itself, at offset (spin ? nu^2 : 0) of the pair's block.
// Dynamic shared memory per warp: n*n double2 (A), n*n double2 (A^-1) when
// Theta is requested, n double2 (pivot reciprocals), n ints (row permutation).
__global__ void overlap_lu_kernel(int N, int nu, int nt, int n, int col0, int spin, long long pairs, int P,
                                  const double* __restrict__ Phi, long long Phi_stride,
                                  const double2* __restrict__ phi, double2* __restrict__ logdet,
                                  double2* __restrict__ Theta, const int* __restrict__ alive, int* status,
                                  int trial_side, double* __restrict__ th2, const int* __restrict__ list,
                                  const int* __restrict__ n_list, int cphi, const dfl* __restrict__ PhiD,
                                  const float4* __restrict__ phiD, int b_df, const float4* __restrict__ Apre) {
    extern __shared__ double2 sm[];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int wpb = blockDim.x >> 5;
    long long pair = (long long)blockIdx.x * wpb + warp;
    if (list) {                                         // only the listed pairs (uniform per warp)
        if (pair >= *n_list) return;
        pair = list[pair];
    }
    if (pair >= pairs) return;
    long long w = pair / P;
    if (alive && !alive[w]) return;
    size_t per_warp = (size_t)n * n * (Theta ? 2 : 1);
    double2* A = sm + warp * (per_warp + n + (n + 1) / 2 + 1);
    double2* Ainv = A + (size_t)n * n;
    double2* dinv = A + per_warp;                       // 1 / u_kk
    int* perm = reinterpret_cast<int*>(dinv + n);
    const double* Ph = Phi + pair * Phi_stride;         // N x nu, spin uses the first n columns
    const double2* ph = phi + w * (long long)N * nt + col0;  // N x nt
    if (n == 0) {
        if (lane == 0) {
            logdet[pair * 2 + spin] = cmk(0.0, 0.0);
            if (th2) th2[pair * 2 + spin] = 0.0;
        }
        return;
    }
    bool bad = false;
    if (Apre) {
        // A formed on the tensor cores (overlap_tc), as double-float entries
        const float4* Ap = Apre + pair * (long long)n * n;
        for (int e = lane; e < n * n; e += 32) {
            const float4 v = Ap[e];
            const double2 t = cmk((double)v.x + (double)v.y, (double)v.z + (double)v.w);
            A[e] = t;
            bad |= !isfinite(t.x) || !isfinite(t.y);
        }
    } else if (PhiD) {
        // double-float products (mixed-precision path, real trial, n <= 64): lane b owns
        // column b0 + b of A (column groups of 32), rows in chunks of 8; Phi entries are
        // broadcast loads, the walker's column one coalesced 16-byte load per row
        const dfl* PD = PhiD + pair * Phi_stride;
        for (int b0 = 0; b0 < n; b0 += 32)
        for (int a0 = 0; a0 < n; a0 += 8) {
            const int b = b0 + lane;
            const float4* pcol = phiD + w * (long long)N * nt + col0 + b;
            float rh[8], rl[8], ih[8], il[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) rh[t] = rl[t] = ih[t] = il[t] = 0.f;
            for (int i = 0; i < N; ++i) {
                const float4 g = b < n ? pcol[(long long)i * nt] : make_float4(0.f, 0.f, 0.f, 0.f);
                const dfl gr = {g.x, g.y}, gi = {g.z, g.w};
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (a0 + t < n) {   // uniform
                        const dfl f = PD[(long long)i * nu + a0 + t];
                        dot2_fma(rh[t], rl[t], f, gr);
                        dot2_fma(ih[t], il[t], f, gi);
                    }
            }
            if (b < n)
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (a0 + t < n) {
                        const double2 v = cmk(df_to(df_two_sum(rh[t], rl[t])), df_to(df_two_sum(ih[t], il[t])));
                        A[(a0 + t) * n + b] = v;
                        bad |= !isfinite(v.x) || !isfinite(v.y);
                    }
        }
    } else
    for (int e = lane; e < n * n; e += 32) {
        int a = e / n, b = e - a * n;
        double2 s = cmk(0.0, 0.0);
        if (cphi) {   // complex trial orbitals: A = Phi^dagger phi
            const double2* Pc = reinterpret_cast<const double2*>(Ph);
            for (int i = 0; i < N; ++i) {
                const double2 f = Pc[(long long)i * nu + a];
                const double2 g = ph[(long long)i * nt + b];
                s.x = fma(f.x, g.x, fma(f.y, g.y, s.x));
                s.y = fma(f.x, g.y, fma(-f.y, g.x, s.y));
            }
        } else {
            for (int i = 0; i < N; ++i) {
                double f = Ph[(long long)i * nu + a];
                double2 g = ph[(long long)i * nt + b];
                s.x = fma(f, g.x, s.x);
                s.y = fma(f, g.y, s.y);
            }
        }
        A[e] = s;
        bad |= !isfinite(s.x) || !isfinite(s.y);
    }
    for (int r = lane; r < n; r += 32) perm[r] = r;
    __syncwarp();
    // orbitals with a non-finite entry have no overlap: NaN log-determinant, so the
    // walker's path signs are NaN and the kill rule removes it
    if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) {
            logdet[pair * 2 + spin] = cmk(__longlong_as_double(0x7FF8000000000000LL), __longlong_as_double(0x7FF8000000000000LL));
            atomicOr(status, STATUS_NONFINITE);
            if (th2) th2[pair * 2 + spin] = INFINITY;
        }
        if (Theta && trial_side == 2) {
            double2* Wp = Theta + pair * (long long)N * nt + (spin ? (long long)nu * nu : 0);
            for (int e = lane; e < n * n; e += 32) Wp[e] = cmk(0.0, 0.0);
        } else if (Theta) {
            double2* Th = Theta + pair * (long long)N * nt + col0;
            for (int e = lane; e < N * n; e += 32) Th[(long long)(e / n) * nt + e % n] = cmk(0.0, 0.0);
        }
        return;
    }
    // The product of the pivots is carried as z * 2^zexp (z rescaled by an exact
    // power of two after every pivot), so log|det| and arg det need one log and
    // one atan2 in all: scalar FP64 work occupies a whole warp instruction.
    double2 z = cmk(1.0, 0.0);
    int zexp = 0;
    bool odd = false;   // odd number of row swaps
    bool singular = false;
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int bi = k;
        for (int r = k + lane; r < n; r += 32) {
            double m = fabs(A[r * n + k].x) + fabs(A[r * n + k].y);
            if (m > best) { best = m; bi = r; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            double ob = __shfl_down_sync(0xffffffffu, best, off);
            int oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        best = __shfl_sync(0xffffffffu, best, 0);
        bi = __shfl_sync(0xffffffffu, bi, 0);
        if (!(best > 0.0)) { singular = true; break; }
        if (bi != k) {
            for (int c = lane; c < n; c += 32) {
                double2 t = A[k * n + c];
                A[k * n + c] = A[bi * n + c];
                A[bi * n + c] = t;
            }
            if (lane == 0) { int t = perm[k]; perm[k] = perm[bi]; perm[bi] = t; }
            odd = !odd;
        }
        __syncwarp();
        const double2 piv = A[k * n + k];
        const double q = 1.0 / fma(piv.x, piv.x, piv.y * piv.y);
        const double2 rinv = cmk(piv.x * q, -piv.y * q);   // 1 / piv
        if (lane == 0) dinv[k] = rinv;
        z = cmul(z, piv);
        {
            const double mz = fmax(fabs(z.x), fabs(z.y));
            int ex = (int)((__double_as_longlong(mz) >> 52) & 0x7FF) - 1023;
            ex = max(-1000, min(1000, ex));
            const double f = __longlong_as_double((long long)(1023 - ex) << 52);   // 2^-ex, exact
            z = cmk(z.x * f, z.y * f);
            zexp += ex;
        }
        for (int r = k + 1 + lane; r < n; r += 32) A[r * n + k] = cmul(A[r * n + k], rinv);
        __syncwarp();
        int m = n - k - 1;
        for (int e = lane; e < m * m; e += 32) {
            int r = k + 1 + e / m, c = k + 1 + e % m;
            double2 t = A[r * n + c];
            double2 l = A[r * n + k], u = A[k * n + c];
            t.x -= l.x * u.x - l.y * u.y;
            t.y -= l.x * u.y + l.y * u.x;
            A[r * n + c] = t;
        }
        __syncwarp();
    }
    if (singular) {
        if (lane == 0) {
            logdet[pair * 2 + spin] = cmk(-INFINITY, 0.0);
            atomicOr(status, STATUS_SINGULAR);
            if (th2) th2[pair * 2 + spin] = INFINITY;
        }
        if (Theta && trial_side == 2) {
            double2* Wp = Theta + pair * (long long)N * nt + (spin ? (long long)nu * nu : 0);
            for (int e = lane; e < n * n; e += 32) Wp[e] = cmk(0.0, 0.0);
        } else if (Theta) {
            double2* Th = Theta + pair * (long long)N * nt + col0;
            for (int e = lane; e < N * n; e += 32) Th[(long long)(e / n) * nt + e % n] = cmk(0.0, 0.0);
        }
        return;
    }
    if (lane == 0) {
        const double logabs = 0.5 * log(fma(z.x, z.x, z.y * z.y)) + zexp * 0.69314718055994530942;
        logdet[pair * 2 + spin] = odd ? cmk(logabs, atan2(-z.y, -z.x)) : cmk(logabs, atan2(z.y, z.x));
    }
    if (!Theta) return;
    // A^-1 column c: solve L y = P e_c (unit lower), then U x = y.
    for (int c = lane; c < n; c += 32) {
        for (int r = 0; r < n; ++r) {
            double2 s = cmk(perm[r] == c ? 1.0 : 0.0, 0.0);
            for (int j = 0; j < r; ++j) {
                double2 l = A[r * n + j], yj = Ainv[j * n + c];
                s.x -= l.x * yj.x - l.y * yj.y;
                s.y -= l.x * yj.y + l.y * yj.x;
            }
            Ainv[r * n + c] = s;
        }
        for (int r = n - 1; r >= 0; --r) {
            double2 s = Ainv[r * n + c];
            for (int j = r + 1; j < n; ++j) {
                double2 u = A[r * n + j], xj = Ainv[j * n + c];
                s.x -= u.x * xj.x - u.y * xj.y;
                s.y -= u.x * xj.y + u.y * xj.x;
            }
            Ainv[r * n + c] = cmul(s, dinv[r]);
        }
    }
    __syncwarp();
    if (th2) {   // ||A^-1||_F^2 (= ||Theta||_F^2 for orthonormal walkers), for the refinement
        double t = 0.0;
        for (int e = lane; e < n * n; e += 32) t = fma(Ainv[e].x, Ainv[e].x, fma(Ainv[e].y, Ainv[e].y, t));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) th2[pair * 2 + spin] = t;
    }
    if (trial_side == 2) {
        // A^-1 itself: pair block [A_up^-1 (nu x nu) | A_dn^-1 (nd x nd)], row-major
        double2* Wp = Theta + pair * (long long)N * nt + (spin ? (long long)nu * nu : 0);
        for (int e = lane; e < n * n; e += 32) Wp[e] = Ainv[e];
        return;
    }
    double2* Th = Theta + pair * (long long)N * nt + col0;
    if (trial_side && b_df) {
        // B = Phi A^-T in double-float, written as (Re hi, Re lo, Im hi, Im lo): A^-1
        // transposed into A's space as double-float values, lane b forms column b of B
        float4* AT = reinterpret_cast<float4*>(A);
        for (int e = lane; e < n * n; e += 32) {
            const int bb = e / n, a = e - bb * n;
            const dfl re = df_from(Ainv[e].x), im = df_from(Ainv[e].y);
            AT[a * n + bb] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
        __syncwarp();
        const dfl* PD = PhiD + pair * Phi_stride;
        for (int b = lane; b < n; b += 32) {
            float4* Bd = reinterpret_cast<float4*>(Th) + b;
            for (int i = 0; i < N; ++i) {
                float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
                for (int a = 0; a < n; ++a) {
                    const dfl f = PD[(long long)i * nu + a];
                    const float4 t = AT[a * n + b];
                    dot2_fma(rh, rl, f, dfl{t.x, t.y});
                    dot2_fma(ih, il, f, dfl{t.z, t.w});
                }
                const dfl re = df_two_sum(rh, rl), im = df_two_sum(ih, il);
                Bd[(long long)i * nt] = make_float4(re.hi, re.lo, im.hi, im.lo);
            }
        }
        return;
    }
    if (trial_side) {
        // B = Phi A^-T (trial side): B[i][b] = sum_a Phi[i][a] (A^-1)[b][a]; for complex
        // trial orbitals B = conj(Phi) A^-T, so that B^T X phi = A^-1 Phi^dagger X phi
        for (int e = lane; e < N * n; e += 32) {
            int i = e / n, b = e - i * n;
            double2 s = cmk(0.0, 0.0);
            if (cphi) {
                const double2* rowc = reinterpret_cast<const double2*>(Ph) + (long long)i * nu;
                for (int a = 0; a < n; ++a) cfma(s, cmk(rowc[a].x, -rowc[a].y), Ainv[b * n + a]);
            } else {
                const double* row = Ph + (long long)i * nu;
                for (int a = 0; a < n; ++a) {
                    const double2 t = Ainv[b * n + a];
                    s.x = fma(row[a], t.x, s.x);
                    s.y = fma(row[a], t.y, s.y);
                }
            }
            Th[(long long)i * nt + b] = s;
        }
        return;
    }
    for (int e = lane; e < N * n; e += 32) {
        int i = e / n, b = e - i * n;
        double2 s = cmk(0.0, 0.0);
        const double2* row = ph + (long long)i * nt;
        for (int a = 0; a < n; ++a) cfma(s, row[a], Ainv[a * n + b]);
        Th[(long long)i * nt + b] = s;
    }
}

static size_t overlap_smem_per_warp(int n, bool theta) {
    return ((size_t)n * n * (theta ? 2 : 1) + n + (n + 1) / 2 + 1) * sizeof(double2);
}

cudaError_t overlap_lu(cudaStream_t s, const Dims& d, int spin, const double* Phi, long long Phi_stride,
                       const double2* phi, double2* logdet, double2* Theta, const int* alive, int* status,
                       long long pairs, int P, int trial_side, double* th2, const int* list, const int* n_list,
                       const void* PhiD, const void* phiD, bool b_df, const void* Apre) {
    // A from the tensor cores: LU, inverse and B in double-float (overlap_lu_df.cu)
    if (Apre && !list && !d.cphi && (!Theta || (trial_side == OVL_TRIAL && b_df)))
        return overlap_lu_df(s, d, spin, Apre, logdet, Theta, alive, status, pairs, P, th2, PhiD, Phi_stride);
    int n = spin == 0 ? d.nu : d.nd;
    if (PhiD && (d.cphi || n > 64 || !phiD)) return cudaErrorInvalidValue;
    if (b_df && (!PhiD || trial_side != OVL_TRIAL)) return cudaErrorInvalidValue;
    int col0 = spin == 0 ? 0 : d.nu;
    size_t per = overlap_smem_per_warp(n, Theta != nullptr);
    int wpb = d.ov_wpb > 0 ? d.ov_wpb : 4;
    while (wpb > 1 && per * wpb > 200 * 1024) wpb >>= 1;
    if (per * wpb > 220 * 1024) return cudaErrorInvalidValue;
    size_t smem = per * wpb;
    cudaError_t e = raise_smem_limit((const void*)overlap_lu_kernel, smem);
    if (e != cudaSuccess) return e;
    long long blocks = (pairs + wpb - 1) / wpb;
    overlap_lu_kernel<<<(unsigned)blocks, 32 * wpb, smem, s>>>(d.N, d.nu, d.nt, n, col0, spin, pairs, P, Phi, Phi_stride,
                                                               phi, logdet, Theta, alive, status, trial_side, th2, list,
                                                               n_list, d.cphi, static_cast<const dfl*>(PhiD),
                                                               static_cast<const float4*>(phiD), b_df ? 1 : 0,
                                                               static_cast<const float4*>(Apre));
    count_launches(1);
    return cudaGetLastError();
}

// Both spins of a pair in one warp, lanes 0-15 on spin up and 16-31 on spin
// down, for n_up <= 16: the same arithmetic as overlap_lu_kernel per spin, but the
// pivot search, the scalar work on each pivot and the column-wise inverse run for
// the two spins at once instead of on 10-odd lanes of a warp each.  Every lane
// reaches every warp synchronisation: a spin with fewer (or no) electrons, or a
// singular overlap, only skips the work of its half.
__global__ void overlap_lu_both_kernel(int N, int nu, int nd, int nt, long long pairs, int P,
                                       const double* __restrict__ Phi, long long Phi_stride,
                                       const double2* __restrict__ phi, double2* __restrict__ logdet,
                                       double2* __restrict__ Theta, const int* __restrict__ alive, int* status,
                                       int trial_side, double* __restrict__ th2, int cphi) {
    extern __shared__ double2 sm[];
    const unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const long long pair = (long long)blockIdx.x * wpb + warp;
    if (pair >= pairs) return;                   // uniform across the warp
    const long long w = pair / P;
    if (alive && !alive[w]) return;              // uniform across the warp
    const int h = lane >> 4, hl = lane & 15;     // half = spin, lane within the half
    const int n = h ? nd : nu, col0 = h ? nu : 0;
    const size_t mats = (size_t)nu * nu * (Theta ? 2 : 1);
    double2* A = sm + (size_t)(warp * 2 + h) * (mats + nu + (nu + 1) / 2 + 1);
    double2* Ainv = A + (size_t)n * n;
    double2* dinv = A + mats;                    // 1 / u_kk
    int* perm = reinterpret_cast<int*>(dinv + nu);
    const double* Ph = Phi + pair * Phi_stride;         // N x nu, spin uses the first n columns
    const double2* ph = phi + w * (long long)N * nt + col0;  // N x nt
    bool bad = false;
    for (int e = hl; e < n * n; e += 16) {
        const int a = e / n, b = e - a * n;
        double2 s = cmk(0.0, 0.0);
        if (cphi) {   // complex trial orbitals: A = Phi^dagger phi
            const double2* Pc = reinterpret_cast<const double2*>(Ph);
            for (int i = 0; i < N; ++i) {
                const double2 f = Pc[(long long)i * nu + a];
                const double2 g = ph[(long long)i * nt + b];
                s.x = fma(f.x, g.x, fma(f.y, g.y, s.x));
                s.y = fma(f.x, g.y, fma(-f.y, g.x, s.y));
            }
        } else {
            for (int i = 0; i < N; ++i) {
                const double f = Ph[(long long)i * nu + a];
                const double2 g = ph[(long long)i * nt + b];
                s.x = fma(f, g.x, s.x);
                s.y = fma(f, g.y, s.y);
            }
        }
        A[e] = s;
        bad |= !isfinite(s.x) || !isfinite(s.y);
    }
    for (int r = hl; r < n; r += 16) perm[r] = r;
    __syncwarp();
    // orbitals with a non-finite entry (either spin) have no overlap: NaN
    // log-determinants, so the walker's path signs are NaN and the kill rule removes it
    if (__any_sync(FULL, bad)) {
        if (hl == 0) {
            logdet[pair * 2 + h] = cmk(__longlong_as_double(0x7FF8000000000000LL), __longlong_as_double(0x7FF8000000000000LL));
            atomicOr(status, STATUS_NONFINITE);
            if (th2) th2[pair * 2 + h] = INFINITY;
        }
        if (Theta && trial_side == 2) {
            double2* Wp = Theta + pair * (long long)N * nt + (h ? (long long)nu * nu : 0);
            for (int e = hl; e < n * n; e += 16) Wp[e] = cmk(0.0, 0.0);
        } else if (Theta) {
            double2* Th = Theta + pair * (long long)N * nt + col0;
            for (int e = hl; e < N * n; e += 16) Th[(long long)(e / n) * nt + e % n] = cmk(0.0, 0.0);
        }
        return;
    }
    double2 z = cmk(1.0, 0.0);
    int zexp = 0;
    bool odd = false;
    bool singular = false;
    for (int k = 0; k < nu; ++k) {               // nu >= nd: the same trip count in both halves
        const bool act = k < n && !singular;     // uniform within a half
        double best = -1.0;
        int bi = k;
        if (act)
            for (int r = k + hl; r < n; r += 16) {
                const double m = fabs(A[r * n + k].x) + fabs(A[r * n + k].y);
                if (m > best) { best = m; bi = r; }
            }
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) {
            const double ob = __shfl_down_sync(FULL, best, off, 16);
            const int oi = __shfl_down_sync(FULL, bi, off, 16);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        best = __shfl_sync(FULL, best, 0, 16);
        bi = __shfl_sync(FULL, bi, 0, 16);
        if (act && !(best > 0.0)) singular = true;
        const bool go = act && !singular;
        if (go && bi != k) {
            for (int c = hl; c < n; c += 16) {
                const double2 t = A[k * n + c];
                A[k * n + c] = A[bi * n + c];
                A[bi * n + c] = t;
            }
            if (hl == 0) { const int t = perm[k]; perm[k] = perm[bi]; perm[bi] = t; }
            odd = !odd;
        }
        __syncwarp();
        if (go) {
            const double2 piv = A[k * n + k];
            const double q = 1.0 / fma(piv.x, piv.x, piv.y * piv.y);
            const double2 rinv = cmk(piv.x * q, -piv.y * q);   // 1 / piv
            if (hl == 0) dinv[k] = rinv;
            z = cmul(z, piv);
            const double mz = fmax(fabs(z.x), fabs(z.y));
            int ex = (int)((__double_as_longlong(mz) >> 52) & 0x7FF) - 1023;
            ex = max(-1000, min(1000, ex));
            const double f = __longlong_as_double((long long)(1023 - ex) << 52);   // 2^-ex, exact
            z = cmk(z.x * f, z.y * f);
            zexp += ex;
            for (int r = k + 1 + hl; r < n; r += 16) A[r * n + k] = cmul(A[r * n + k], rinv);
        }
        __syncwarp();
        if (go) {
            const int m = n - k - 1;
            for (int e = hl; e < m * m; e += 16) {
                const int r = k + 1 + e / m, c = k + 1 + e % m;
                double2 t = A[r * n + c];
                const double2 l = A[r * n + k], u = A[k * n + c];
                t.x -= l.x * u.x - l.y * u.y;
                t.y -= l.x * u.y + l.y * u.x;
                A[r * n + c] = t;
            }
        }
        __syncwarp();
    }
    if (n == 0) {
        if (hl == 0) logdet[pair * 2 + h] = cmk(0.0, 0.0);
    } else if (singular) {
        if (hl == 0) {
            logdet[pair * 2 + h] = cmk(-INFINITY, 0.0);
            atomicOr(status, STATUS_SINGULAR);
        }
        if (Theta && trial_side == 2) {
            double2* Wp = Theta + pair * (long long)N * nt + (h ? (long long)nu * nu : 0);
            for (int e = hl; e < n * n; e += 16) Wp[e] = cmk(0.0, 0.0);
        } else if (Theta) {
            double2* Th = Theta + pair * (long long)N * nt + col0;
            for (int e = hl; e < N * n; e += 16) Th[(long long)(e / n) * nt + e % n] = cmk(0.0, 0.0);
        }
    } else if (hl == 0) {
        const double logabs = 0.5 * log(fma(z.x, z.x, z.y * z.y)) + zexp * 0.69314718055994530942;
        logdet[pair * 2 + h] = odd ? cmk(logabs, atan2(-z.y, -z.x)) : cmk(logabs, atan2(z.y, z.x));
    }
    if (!Theta) return;                          // uniform: a kernel argument
    const bool inv = n > 0 && !singular;
    // A^-1 column c: solve L y = P e_c (unit lower), then U x = y.
    if (inv)
        for (int c = hl; c < n; c += 16) {
            for (int r = 0; r < n; ++r) {
                double2 s = cmk(perm[r] == c ? 1.0 : 0.0, 0.0);
                for (int j = 0; j < r; ++j) {
                    const double2 l = A[r * n + j], yj = Ainv[j * n + c];
                    s.x -= l.x * yj.x - l.y * yj.y;
                    s.y -= l.x * yj.y + l.y * yj.x;
                }
                Ainv[r * n + c] = s;
            }
            for (int r = n - 1; r >= 0; --r) {
                double2 s = Ainv[r * n + c];
                for (int j = r + 1; j < n; ++j) {
                    const double2 u = A[r * n + j], xj = Ainv[j * n + c];
                    s.x -= u.x * xj.x - u.y * xj.y;
                    s.y -= u.x * xj.y + u.y * xj.x;
                }
                Ainv[r * n + c] = cmul(s, dinv[r]);
            }
        }
    __syncwarp();
    if (th2) {   // ||A^-1||_F^2 per spin (every lane takes part in the half-warp sums)
        double t = 0.0;
        if (inv)
            for (int e = hl; e < n * n; e += 16) t = fma(Ainv[e].x, Ainv[e].x, fma(Ainv[e].y, Ainv[e].y, t));
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) t += __shfl_xor_sync(FULL, t, off);
        if (hl == 0) th2[pair * 2 + h] = n == 0 ? 0.0 : (inv ? t : INFINITY);
    }
    if (!inv) return;                            // nothing below synchronises the warp
    if (trial_side == 2) {
        double2* Wp = Theta + pair * (long long)N * nt + (h ? (long long)nu * nu : 0);
        for (int e = hl; e < n * n; e += 16) Wp[e] = Ainv[e];
        return;
    }
    double2* Th = Theta + pair * (long long)N * nt + col0;
    if (trial_side) {   // B = Phi A^-T, or conj(Phi) A^-T for complex trial orbitals
        for (int e = hl; e < N * n; e += 16) {
            const int i = e / n, b = e - i * n;
            double2 s = cmk(0.0, 0.0);
            if (cphi) {
                const double2* rowc = reinterpret_cast<const double2*>(Ph) + (long long)i * nu;
                for (int a = 0; a < n; ++a) cfma(s, cmk(rowc[a].x, -rowc[a].y), Ainv[b * n + a]);
            } else {
                const double* row = Ph + (long long)i * nu;
                for (int a = 0; a < n; ++a) {
                    const double2 t = Ainv[b * n + a];
                    s.x = fma(row[a], t.x, s.x);
                    s.y = fma(row[a], t.y, s.y);
                }
            }
            Th[(long long)i * nt + b] = s;
        }
        return;
    }
    for (int e = hl; e < N * n; e += 16) {
        const int i = e / n, b = e - i * n;
        double2 s = cmk(0.0, 0.0);
        const double2* row = ph + (long long)i * nt;
        for (int a = 0; a < n; ++a) cfma(s, row[a], Ainv[a * n + b]);
        Th[(long long)i * nt + b] = s;
    }
}

cudaError_t overlap_lu_both(cudaStream_t s, const Dims& d, const double* Phi, long long Phi_stride,
                            const double2* phi, double2* logdet, double2* Theta, const int* alive, int* status,
                            long long pairs, int P, int trial_side, double* th2, const void* PhiD, const void* phiD,
                            bool b_df, const void* Apre) {
    // a half-warp per spin would leave the larger matrices short of lanes; the
    // double-float products run in the per-spin kernel
    if (d.nu > 16 || PhiD || Apre) {
        for (int spin = 0; spin < 2; ++spin) {
            const void* Ap = Apre ? static_cast<const float4*>(Apre) + (spin ? d.pairs * (long long)d.nu * d.nu : 0)
                                  : nullptr;
            const cudaError_t e = overlap_lu(s, d, spin, Phi, Phi_stride, phi, logdet, Theta, alive, status, pairs, P,
                                             trial_side, th2, nullptr, nullptr, PhiD, phiD, b_df, Ap);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (pairs <= 0) return cudaSuccess;
    const size_t per = 2 * ((size_t)d.nu * d.nu * (Theta ? 2 : 1) + d.nu + (d.nu + 1) / 2 + 1) * sizeof(double2);
    int wpb = d.ov_wpb > 0 ? d.ov_wpb : 4;
    while (wpb > 1 && per * wpb > 200 * 1024) wpb >>= 1;
    const size_t smem = per * wpb;
    cudaError_t e = raise_smem_limit((const void*)overlap_lu_both_kernel, smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (pairs + wpb - 1) / wpb;
    overlap_lu_both_kernel<<<(unsigned)blocks, 32 * wpb, smem, s>>>(d.N, d.nu, d.nd, d.nt, pairs, P, Phi, Phi_stride,
                                                                    phi, logdet, Theta, alive, status, trial_side, th2,
                                                                    d.cphi);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- re-orthonormalisation
// One warp per (walker, spin): modified Gram-Schmidt on the N x n complex
// block (columns col0..), q_j = (v_j - sum_k<j (q_k^H v_j) q_k) / norm, so
// phi = Q R with R upper triangular and diag(R) > 0.  Dead walkers are copied.
__global__ void reorth_kernel(int N, int nt, int n, int col0, const double2* __restrict__ src, double2* __restrict__ dst,
                              const int* __restrict__ alive, int* status) {
    extern __shared__ double2 q[];   // N x n
    long long w = blockIdx.x;
    int lane = threadIdx.x;
    const double2* in = src + w * (long long)N * nt + col0;
    double2* out = dst + w * (long long)N * nt + col0;
    for (int e = lane; e < N * n; e += 32) q[e] = in[(long long)(e / n) * nt + e % n];
    __syncwarp();
    if (alive == nullptr || alive[w]) {
        for (int j = 0; j < n; ++j) {
            for (int k = 0; k < j; ++k) {
                double2 dot = cmk(0.0, 0.0);
                for (int i = lane; i < N; i += 32) cfma(dot, cconj(q[i * n + k]), q[i * n + j]);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    dot.x += __shfl_xor_sync(0xffffffffu, dot.x, off);
                    dot.y += __shfl_xor_sync(0xffffffffu, dot.y, off);
                }
                for (int i = lane; i < N; i += 32) {
                    double2 v = q[i * n + j], qk = q[i * n + k];
                    v.x -= dot.x * qk.x - dot.y * qk.y;
                    v.y -= dot.x * qk.y + dot.y * qk.x;
                    q[i * n + j] = v;
                }
                __syncwarp();
            }
            double nrm = 0.0;
            for (int i = lane; i < N; i += 32) nrm += q[i * n + j].x * q[i * n + j].x + q[i * n + j].y * q[i * n + j].y;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
            if (!(nrm > 0.0) || !isfinite(nrm)) {
                if (lane == 0) atomicOr(status, STATUS_NONFINITE);
                nrm = 1.0;
            }
            double inv = 1.0 / sqrt(nrm);
            for (int i = lane; i < N; i += 32) q[i * n + j] = cscale(q[i * n + j], inv);
            __syncwarp();
        }
    }
    for (int e = lane; e < N * n; e += 32) out[(long long)(e / n) * nt + e % n] = q[e];
}

cudaError_t reorthonormalise(cudaStream_t s, const Dims& d, const double2* src, double2* dst, const int* alive, int* status,
                             int n_walkers) {
    for (int spin = 0; spin < 2; ++spin) {
        int n = spin == 0 ? d.nu : d.nd;
        if (n == 0) continue;
        size_t smem = (size_t)d.N * n * sizeof(double2);
        cudaError_t e = raise_smem_limit((const void*)reorth_kernel, smem);
        if (e != cudaSuccess) return e;
        reorth_kernel<<<n_walkers, 32, smem, s>>>(d.N, d.nt, n, spin == 0 ? 0 : d.nu, src, dst, alive, status); count_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- trial orbitals
// Phi = exp(S) Phi0 for one symmetric S per problem, by the Chebyshev series
// exp(c + rho t) = e^c [I_0(rho) + 2 sum_k I_k(rho) T_k(t)] on the Gershgorin
// interval [c - rho, c + rho] of S, with modified Bessel I_k from Miller's
// backward recurrence, truncated once the remaining coefficients fall below
// 1e-18 of e^rho.  One block per problem; S in shared memory when it fits.
constexpr int CHEB_MAX = 320;

template <bool S_SMEM>
__global__ void __launch_bounds__(256) chebyshev_expm_kernel(int N, int nu, long long problems, const double* __restrict__ S_all,
                                                             const double* __restrict__ Phi0, double* __restrict__ Out,
                                                             const int* __restrict__ alive, int P, int* status) {
    extern __shared__ double smd[];
    __shared__ double coef[CHEB_MAX + 2];
    __shared__ double red_lo[256], red_hi[256];
    __shared__ int nterms;
    __shared__ double cshift, rho_s;
    long long prob = blockIdx.x;
    if (alive && !alive[prob / P]) return;
    const double* Sg = S_all + prob * (long long)N * N;
    double* S = S_SMEM ? smd : nullptr;
    double* Vp = S_SMEM ? smd + (size_t)N * N : smd;
    double* Vc = Vp + (size_t)N * nu;
    double* acc = Vc + (size_t)N * nu;
    int tid = threadIdx.x, nth = blockDim.x;
    if (S_SMEM)
        for (int e = tid; e < N * N; e += nth) S[e] = Sg[e];
    __syncthreads();
    const double* Sr = S_SMEM ? S : Sg;
    double lo = INFINITY, hi = -INFINITY;
    for (int i = tid; i < N; i += nth) {
        double r = 0.0;
        for (int j = 0; j < N; ++j)
            if (j != i) r += fabs(Sr[(long long)i * N + j]);
        lo = fmin(lo, Sr[(long long)i * N + i] - r);
        hi = fmax(hi, Sr[(long long)i * N + i] + r);
    }
    red_lo[tid] = lo;
    red_hi[tid] = hi;
    __syncthreads();
    for (int off = nth / 2; off > 0; off >>= 1) {
        if (tid < off) {
            red_lo[tid] = fmin(red_lo[tid], red_lo[tid + off]);
            red_hi[tid] = fmax(red_hi[tid], red_hi[tid + off]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        double c = 0.5 * (red_lo[0] + red_hi[0]);
        double rho = fmax(0.5 * (red_hi[0] - red_lo[0]), 1e-3);
        int start = (int)ceil(rho) + 48;
        if (!isfinite(rho) || start > CHEB_MAX) {
            atomicOr(status, STATUS_NONFINITE);
            start = CHEB_MAX;
        }
        // Miller: I_{k-1} = (2k / rho) I_k + I_{k+1}, started at order `start` with I = 0, 1.
        double ip1 = 0.0, ik = 1e-280;
        for (int k = start; k >= 1; --k) {
            coef[k] = ik;
            double im1 = (2.0 * k / rho) * ik + ip1;
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
        double lscale = c + rho - log(norm);
        coef[0] = exp(lscale + log(coef[0]));
        for (int k = 1; k <= m; ++k) coef[k] = 2.0 * exp(lscale + log(coef[k]));
        nterms = m;
        cshift = c;
        rho_s = rho;
    }
    __syncthreads();
    int m = nterms;
    double c = cshift, irho = 1.0 / rho_s;
    int nn = N * nu;
    for (int e = tid; e < nn; e += nth) {
        Vp[e] = Phi0[e];
        acc[e] = coef[0] * Phi0[e];
    }
    __syncthreads();
    // V1 = t Phi0 with t = (S - c) / rho
    for (int e = tid; e < nn; e += nth) {
        int i = e / nu, a = e - i * nu;
        double s = 0.0;
        for (int j = 0; j < N; ++j) s = fma(Sr[(long long)i * N + j], Vp[j * nu + a], s);
        s = (s - c * Vp[e]) * irho;
        Vc[e] = s;
        acc[e] = fma(coef[1], s, acc[e]);
    }
    __syncthreads();
    for (int k = 2; k <= m; ++k) {
        // V_k = 2 t V_{k-1} - V_{k-2}.  Element e of V_k needs all of V_{k-1} (Vc)
        // but only element e of V_{k-2} (Vp), so it overwrites Vp[e] in place.
        for (int e = tid; e < nn; e += nth) {
            int i = e / nu, a = e - i * nu;
            double s = 0.0;
            for (int j = 0; j < N; ++j) s = fma(Sr[(long long)i * N + j], Vc[j * nu + a], s);
            s = (s - c * Vc[e]) * irho;
            double v = 2.0 * s - Vp[e];
            Vp[e] = v;
            acc[e] = fma(coef[k], v, acc[e]);
        }
        __syncthreads();
        double* t = Vp; Vp = Vc; Vc = t;
    }
    double* o = Out + prob * (long long)nn;
    for (int e = tid; e < nn; e += nth) o[e] = acc[e];
}

cudaError_t trial_orbitals_gershgorin(cudaStream_t s, int N, int nu, long long problems, const double* S_all,
                                      const double* Phi0, double* Out, const int* alive, int P, int* status, int threads) {
    if (problems <= 0) return cudaSuccess;
    if (threads != 128 && threads != 256) threads = 256;
    size_t vec = 3 * (size_t)N * nu * sizeof(double);
    size_t full = vec + (size_t)N * N * sizeof(double);
    cudaError_t e;
    if (full <= 200 * 1024) {
        e = raise_smem_limit((const void*)chebyshev_expm_kernel<true>, full);
        if (e != cudaSuccess) return e;
        chebyshev_expm_kernel<true><<<(unsigned)problems, threads, full, s>>>(N, nu, problems, S_all, Phi0, Out, alive, P, status); count_launches(1);
    } else {
        if (vec > 200 * 1024) return cudaErrorInvalidValue;
        e = raise_smem_limit((const void*)chebyshev_expm_kernel<false>, vec);
        if (e != cudaSuccess) return e;
        chebyshev_expm_kernel<false><<<(unsigned)problems, threads, vec, s>>>(N, nu, problems, S_all, Phi0, Out, alive, P, status); count_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- init: T and exp(-tau T / 2)
// T = h - 1/2 sum_g L_g L_g (Monte Carlo form of the Hamiltonian).
__global__ void one_body_T_kernel(int N, int G, const double* __restrict__ h, const double* __restrict__ L, double* T) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)N * N) return;
    int i = (int)(e / N), k = (int)(e % N);
    double s = 0.0;
    for (int g = 0; g < G; ++g) {
        const double* Lg = L + (long long)g * N * N;
        for (int j = 0; j < N; ++j) s = fma(Lg[(long long)i * N + j], Lg[(long long)j * N + k], s);
    }
    T[e] = h[e] - 0.5 * s;
}

// exp(alpha * T) by scaling and squaring with a degree-20 Taylor polynomial in
// Horner form; one block, matrices in global scratch X, E, Y (N*N each).
__global__ void __launch_bounds__(1024) expm_small_kernel(int N, double alpha, const double* __restrict__ T, double* X,
                                                          double* E, double* Y, double* out) {
    __shared__ double red[1024];
    __shared__ int s_sq;
    int tid = threadIdx.x, nth = blockDim.x;
    long long NN = (long long)N * N;
    double colmax = 0.0;
    for (int j = tid; j < N; j += nth) {
        double cs = 0.0;
        for (int i = 0; i < N; ++i) cs += fabs(alpha * T[(long long)i * N + j]);
        colmax = fmax(colmax, cs);
    }
    red[tid] = colmax;
    __syncthreads();
    for (int off = nth / 2; off > 0; off >>= 1) {
        if (tid < off) red[tid] = fmax(red[tid], red[tid + off]);
        __syncthreads();
    }
    if (tid == 0) {
        int sq = 0;
        double nrm = red[0];
        while (nrm > 0.5 && sq < 60) { nrm *= 0.5; ++sq; }
        s_sq = sq;
    }
    __syncthreads();
    int sq = s_sq;
    double scale = alpha * ldexp(1.0, -sq);
    for (long long e = tid; e < NN; e += nth) {
        X[e] = scale * T[e];
        E[e] = ((e / N) == (e % N)) ? 1.0 : 0.0;
    }
    __syncthreads();
    // Horner: E = I + X/q (I + X/(q-1) ( ... )) with q from 20 down to 1
    for (int q = 20; q >= 1; --q) {
        for (long long e = tid; e < NN; e += nth) {
            int i = (int)(e / N), k = (int)(e % N);
            double s = 0.0;
            for (int j = 0; j < N; ++j) s = fma(X[(long long)i * N + j], E[(long long)j * N + k], s);
            Y[e] = (i == k ? 1.0 : 0.0) + s / q;
        }
        __syncthreads();
        for (long long e = tid; e < NN; e += nth) E[e] = Y[e];
        __syncthreads();
    }
    for (int r = 0; r < sq; ++r) {
        for (long long e = tid; e < NN; e += nth) {
            int i = (int)(e / N), k = (int)(e % N);
            double s = 0.0;
            for (int j = 0; j < N; ++j) s = fma(E[(long long)i * N + j], E[(long long)j * N + k], s);
            Y[e] = s;
        }
        __syncthreads();
        for (long long e = tid; e < NN; e += nth) E[e] = Y[e];
        __syncthreads();
    }
    for (long long e = tid; e < NN; e += nth) out[e] = E[e];
}

cudaError_t one_body_propagator(cudaStream_t s, int N, int G, double dtau, const double* h, const double* L, double* T,
                                double* scratch3, double* expT) {
    long long NN = (long long)N * N;
    one_body_T_kernel<<<(unsigned)((NN + 127) / 128), 128, 0, s>>>(N, G, h, L, T); count_launches(1);
    expm_small_kernel<<<1, 1024, 0, s>>>(N, -0.5 * dtau, T, scratch3, scratch3 + NN, scratch3 + 2 * NN, expT); count_launches(1);
    return cudaGetLastError();
}

}  // namespace afq
