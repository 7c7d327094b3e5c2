// Complex and multi-slice trial samples (FP64 path): the single-slice VAFQMC
// form Phi(x) = exp(alpha sum_k x_k U_k) Phi0 with a complex alpha (Eq. (30);
// alpha = -i sqrt(s) and U_k = L_k there), and the multi-slice form
//   Phi(x) = exp(alpha S_m) P ... P exp(alpha S_1) Phi0,  S_l = sum_k x_lk U_k,
// with a fixed real propagator P between slices (Eq. (19), (32)).  Overlaps and
// Green's functions then take Phi^dagger (the overlap and contraction kernels
// read Phi as complex).
//
// exp(alpha S) V for real symmetric S: with the Gershgorin interval
// [c - rho, c + rho] of S and t = (S - c) / rho,
//   exp(alpha S) = e^(alpha c) [I_0(z) + 2 sum_k I_k(z) T_k(t)],  z = alpha rho,
// the modified Bessel functions of the complex argument z by Miller's backward
// recurrence I_(k-1) = (2k / z) I_k + I_(k+1), normalised by
// I_0 + 2 sum_k I_k = e^z (for imaginary z this is the usual recurrence of J_k,
// I_k(iy) = i^k J_k(y)).  The Chebyshev vectors T_k(t) V stay real when V is
// real; only the coefficients are complex.
#include "kernels.cuh"

namespace afq {

constexpr int CHEB_C_MAX = 512;

__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Coefficients a_k = (2 - delta_k0) I_k(z) e^(alpha c), k <= m; returns m.  One thread.
__device__ int cheb_coefs_c(double2 alpha, double c, double rho, double2* coef, int* status) {
    const double2 z = cmul(alpha, cmk(rho, 0.0));
    const double az = sqrt(cabs2(z));
    int start = (int)ceil(az) + 48;
    if (!isfinite(az) || start > CHEB_C_MAX) {
        atomicOr(status, STATUS_NONFINITE);
        start = CHEB_C_MAX;
    }
    // 2 / z
    const double iz2 = 1.0 / fmax(cabs2(z), 1e-300);
    const double2 r2 = cmk(2.0 * z.x * iz2, -2.0 * z.y * iz2);
    double2 ip1 = cmk(0.0, 0.0), ik = cmk(1e-280, 0.0);
    for (int k = start; k >= 1; --k) {
        coef[k] = ik;
        const double2 im1 = cadd(cmul(cscale(r2, (double)k), ik), ip1);
        ip1 = ik;
        ik = im1;
        if (fabs(ik.x) > 1e250 || fabs(ik.y) > 1e250) {   // rescale everything computed so far
            for (int j = k; j <= start; ++j) coef[j] = cscale(coef[j], 1e-250);
            ip1 = cscale(ip1, 1e-250);
            ik = cscale(ik, 1e-250);
        }
    }
    coef[0] = ik;
    double2 norm = coef[0];
    double mag = sqrt(cabs2(coef[0]));
    for (int k = 1; k <= start; ++k) {
        norm = cadd(norm, cscale(coef[k], 2.0));
        mag += 2.0 * sqrt(cabs2(coef[k]));
    }
    int m = start;
    for (int k = 1; k <= start; ++k)
        if (sqrt(cabs2(coef[k])) < 1e-18 * mag && k > az) { m = k; break; }
    // scale: e^(z + alpha c) / norm
    const double2 ez = cexp_(cadd(z, cmul(alpha, cmk(c, 0.0))));
    const double2 sc = cdiv(ez, norm);
    coef[0] = cmul(coef[0], sc);
    for (int k = 1; k <= m; ++k) coef[k] = cscale(cmul(coef[k], sc), 2.0);
    return m;
}

// One block per problem: Out = exp(alpha S) V0 (N x nu complex), S = S_all[prob]
// (real symmetric N x N), V0 = Phi0 (real, the same for every problem) or
// Vin[prob] (complex).  Shared memory: S (when S_SMEM), and three complex
// N x nu arrays (V_(k-1), V_k, the sum).
template <bool S_SMEM, bool V0_REAL>
__global__ void __launch_bounds__(256) chebyshev_expm_c_kernel(int N, int nu, long long problems,
                                                               const double* __restrict__ S_all, double2 alpha,
                                                               const double* __restrict__ Phi0,
                                                               const double2* __restrict__ Vin, double2* __restrict__ Out,
                                                               const int* __restrict__ alive, int P, int* status) {
    extern __shared__ double smd[];
    __shared__ double2 coef[CHEB_C_MAX + 2];
    __shared__ double red_lo[256], red_hi[256];
    __shared__ int nterms;
    __shared__ double cshift, rho_s;
    const long long prob = blockIdx.x;
    if (alive && !alive[prob / P]) return;
    const double* Sg = S_all + prob * (long long)N * N;
    double* S = S_SMEM ? smd : nullptr;
    // the complex arrays start on a 16-byte boundary: S takes N*N doubles rounded up to even
    double2* Vp = reinterpret_cast<double2*>(S_SMEM ? smd + (((size_t)N * N + 1) & ~(size_t)1) : smd);
    double2* Vc = Vp + (size_t)N * nu;
    double2* acc = Vc + (size_t)N * nu;
    const int tid = threadIdx.x, nth = blockDim.x;
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
        const double c = 0.5 * (red_lo[0] + red_hi[0]);
        const double rho = fmax(0.5 * (red_hi[0] - red_lo[0]), 1e-3);
        nterms = cheb_coefs_c(alpha, c, rho, coef, status);
        cshift = c;
        rho_s = rho;
    }
    __syncthreads();
    const int m = nterms;
    const double c = cshift, irho = 1.0 / rho_s;
    const int nn = N * nu;
    const double2* vin = V0_REAL ? nullptr : Vin + prob * (long long)nn;
    for (int e = tid; e < nn; e += nth) {
        const double2 v = V0_REAL ? cmk(Phi0[e], 0.0) : vin[e];
        Vp[e] = v;
        acc[e] = cmul(coef[0], v);
    }
    __syncthreads();
    // V_1 = t V_0
    for (int e = tid; e < nn; e += nth) {
        const int i = e / nu, a = e - i * nu;
        double2 s = cmk(0.0, 0.0);
        for (int j = 0; j < N; ++j) {
            const double sij = Sr[(long long)i * N + j];
            const double2 v = Vp[j * nu + a];
            s.x = fma(sij, v.x, s.x);
            s.y = fma(sij, v.y, s.y);
        }
        s = cscale(csub(s, cscale(Vp[e], c)), irho);
        Vc[e] = s;
        cfma(acc[e], coef[1], s);
    }
    __syncthreads();
    for (int k = 2; k <= m; ++k) {
        // V_k = 2 t V_(k-1) - V_(k-2), written over V_(k-2) element by element
        for (int e = tid; e < nn; e += nth) {
            const int i = e / nu, a = e - i * nu;
            double2 s = cmk(0.0, 0.0);
            for (int j = 0; j < N; ++j) {
                const double sij = Sr[(long long)i * N + j];
                const double2 v = Vc[j * nu + a];
                s.x = fma(sij, v.x, s.x);
                s.y = fma(sij, v.y, s.y);
            }
            s = cscale(csub(s, cscale(Vc[e], c)), irho);
            const double2 v = csub(cscale(s, 2.0), Vp[e]);
            Vp[e] = v;
            cfma(acc[e], coef[k], v);
        }
        __syncthreads();
        double2* t = Vp;
        Vp = Vc;
        Vc = t;
    }
    double2* o = Out + prob * (long long)nn;
    for (int e = tid; e < nn; e += nth) o[e] = acc[e];
}

bool trial_orbitals_c_supported(int N, int nu) { return 3 * (size_t)N * nu * sizeof(double2) <= 200 * 1024; }

cudaError_t trial_orbitals_c(cudaStream_t s, int N, int nu, long long problems, const double* S_all, double2 alpha,
                             const double* Phi0, const double2* Vin, double2* Out, const int* alive, int P,
                             int* status) {
    if (problems <= 0) return cudaSuccess;
    const size_t vec = 3 * (size_t)N * nu * sizeof(double2);
    const size_t full = vec + (((size_t)N * N + 1) & ~(size_t)1) * sizeof(double);
    if (vec > 200 * 1024) return cudaErrorInvalidValue;
    const bool s_smem = full <= 200 * 1024;
    const size_t smem = s_smem ? full : vec;
    const void* k = s_smem ? (Vin ? (const void*)chebyshev_expm_c_kernel<true, false>
                                  : (const void*)chebyshev_expm_c_kernel<true, true>)
                           : (Vin ? (const void*)chebyshev_expm_c_kernel<false, false>
                                  : (const void*)chebyshev_expm_c_kernel<false, true>);
    cudaError_t e = raise_smem_limit(k, smem);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)problems;
    if (s_smem && Vin)
        chebyshev_expm_c_kernel<true, false><<<g, 256, smem, s>>>(N, nu, problems, S_all, alpha, Phi0, Vin, Out, alive, P, status);
    else if (s_smem)
        chebyshev_expm_c_kernel<true, true><<<g, 256, smem, s>>>(N, nu, problems, S_all, alpha, Phi0, Vin, Out, alive, P, status);
    else if (Vin)
        chebyshev_expm_c_kernel<false, false><<<g, 256, smem, s>>>(N, nu, problems, S_all, alpha, Phi0, Vin, Out, alive, P, status);
    else
        chebyshev_expm_c_kernel<false, true><<<g, 256, smem, s>>>(N, nu, problems, S_all, alpha, Phi0, Vin, Out, alive, P, status);
    count_launches(1);
    return cudaGetLastError();
}

// Out[prob] = Pm V[prob] (Pm real N x N, V complex N x nu), one block per problem.
__global__ void __launch_bounds__(256) slice_propagate_kernel(int N, int nu, const double* __restrict__ Pm,
                                                              const double2* __restrict__ V, double2* __restrict__ Out,
                                                              const int* __restrict__ alive, int P) {
    const long long prob = blockIdx.x;
    if (alive && !alive[prob / P]) return;
    const double2* v = V + prob * (long long)N * nu;
    double2* o = Out + prob * (long long)N * nu;
    for (int e = threadIdx.x; e < N * nu; e += blockDim.x) {
        const int i = e / nu, a = e - i * nu;
        double2 s = cmk(0.0, 0.0);
        for (int j = 0; j < N; ++j) {
            const double p = Pm[(long long)i * N + j];
            const double2 x = v[j * nu + a];
            s.x = fma(p, x.x, s.x);
            s.y = fma(p, x.y, s.y);
        }
        o[e] = s;
    }
}

cudaError_t slice_propagate(cudaStream_t s, int N, int nu, long long problems, const double* Pm, const double2* V,
                            double2* Out, const int* alive, int P) {
    if (problems <= 0) return cudaSuccess;
    slice_propagate_kernel<<<(unsigned)problems, 256, 0, s>>>(N, nu, Pm, V, Out, alive, P);
    count_launches(1);
    return cudaGetLastError();
}

// phi_w = Phi(x_w) for both spins (spin down: the first n_dn columns), from
// complex trial orbitals.
__global__ void walkers_from_trial_c_kernel(int N, int nu, int nd, const double2* __restrict__ Phi_w, double2* phi) {
    const long long w = blockIdx.x;
    const int nt = nu + nd;
    for (int e = threadIdx.x; e < N * nt; e += blockDim.x) {
        const int i = e / nt, c = e - i * nt;
        const int src = c < nu ? c : c - nu;
        phi[w * (long long)N * nt + e] = Phi_w[w * (long long)N * nu + (long long)i * nu + src];
    }
}

cudaError_t walkers_from_trial_c(cudaStream_t s, const Dims& d, const double2* Phi_w, double2* phi) {
    walkers_from_trial_c_kernel<<<d.W, 128, 0, s>>>(d.N, d.nu, d.nd, Phi_w, phi);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace afq

namespace afq {

// ---------------------------------------------------------------- contraction with complex Phi
// The per-pair FP64 contraction of Eq. (15), (16), (27) for complex trial
// orbitals: R_g = Phi^dagger X_g (n_up x N, complex), M_g,s = R_g[:n_s] Theta_s,
// v_g = sum_s Tr M_g,s, E_L = sum_s Tr M_h,s + 1/2 sum_g [v_g^2 - sum_s Tr M_g,s^2].
// One block per pair; Phi and Theta in shared memory, column blocks of X_g
// streamed; each thread owns up to CC_OWN entries of the two M blocks.
constexpr int CC_T = 256, CC_OWN = 16, CC_JB = 16;

__device__ __forceinline__ double2 cc_block_sum(double2 v, double2* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double2 t = cmk(0.0, 0.0);
    if (threadIdx.x < 32) {
        t = lane < CC_T / 32 ? red[lane] : cmk(0.0, 0.0);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            t.x += __shfl_xor_sync(0xffffffffu, t.x, off);
            t.y += __shfl_xor_sync(0xffffffffu, t.y, off);
        }
    }
    __syncthreads();
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(CC_T) contract_fp64c_kernel(int N, int nu, int nd, int G, const double* __restrict__ h,
                                                              const double* __restrict__ L,
                                                              const double2* __restrict__ Phi,
                                                              const double2* __restrict__ Theta,
                                                              double2* __restrict__ vpair, double2* __restrict__ epair,
                                                              const int* __restrict__ list, const int* __restrict__ n_list) {
    extern __shared__ double2 scc[];
    __shared__ double2 red[CC_T / 32];
    const int nt = nu + nd, tid = threadIdx.x;
    const int nM = nu * nu + nd * nd;
    double2* sPhi = scc;                               // N x nu
    double2* sTh = sPhi + (size_t)N * nu;              // N x nt
    double2* sR = sTh + (size_t)N * nt;                // nu x CC_JB
    double2* sM = sR + (size_t)nu * CC_JB;             // nM
    double* sL = reinterpret_cast<double*>(sM + nM);   // N x CC_JB
    long long pair = blockIdx.x;
    if (list) {   // only the listed pairs (uniform per block)
        if (pair >= *n_list) return;
        pair = list[pair];
    }
    const double2* gPhi = Phi + pair * (long long)N * nu;
    const double2* gTh = Theta + pair * (long long)N * nt;
    for (int e = tid; e < N * nu; e += CC_T) sPhi[e] = gPhi[e];
    for (int e = tid; e < N * nt; e += CC_T) sTh[e] = gTh[e];
    int own_a[CC_OWN], own_b[CC_OWN], own_c[CC_OWN], nown = 0;
#pragma unroll
    for (int r = 0; r < CC_OWN; ++r) {
        const int o = tid + r * CC_T;
        own_a[r] = own_b[r] = own_c[r] = 0;
        if (o >= nM) continue;
        nown = r + 1;
        if (o < nu * nu) { own_a[r] = o / nu; own_b[r] = o % nu; own_c[r] = o % nu; }
        else { const int q = o - nu * nu; own_a[r] = q / nd; own_b[r] = q % nd; own_c[r] = nu + q % nd; }
    }
    double2 e_acc = cmk(0.0, 0.0);
    __syncthreads();
    for (int g = -1; g < G; ++g) {
        const double* Xg = g < 0 ? h : L + (long long)g * N * N;
        double2 acc[CC_OWN];
#pragma unroll
        for (int r = 0; r < CC_OWN; ++r) acc[r] = cmk(0.0, 0.0);
        for (int j0 = 0; j0 < N; j0 += CC_JB) {
            const int jb = min(CC_JB, N - j0);
            for (int e = tid; e < N * jb; e += CC_T) {
                const int i = e / jb, j = e - i * jb;
                sL[i * CC_JB + j] = Xg[(long long)i * N + j0 + j];
            }
            __syncthreads();
            // R[a, j] = sum_i conj(Phi[i, a]) X[i, j0 + j]
            for (int e = tid; e < nu * jb; e += CC_T) {
                const int a = e / jb, j = e - a * jb;
                double2 sr = cmk(0.0, 0.0);
                for (int i = 0; i < N; ++i) {
                    const double2 f = sPhi[i * nu + a];
                    const double x = sL[i * CC_JB + j];
                    sr.x = fma(f.x, x, sr.x);
                    sr.y = fma(-f.y, x, sr.y);
                }
                sR[a * CC_JB + j] = sr;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < CC_OWN; ++r) {
                if (r >= nown) break;
                const double2* Ra = sR + own_a[r] * CC_JB;
                const double2* Tc = sTh + (size_t)j0 * nt + own_c[r];
                double2 s = acc[r];
                for (int j = 0; j < jb; ++j) cfma(s, Ra[j], Tc[(size_t)j * nt]);
                acc[r] = s;
            }
            __syncthreads();
        }
        double2 tr = cmk(0.0, 0.0);
#pragma unroll
        for (int r = 0; r < CC_OWN; ++r) {
            if (r >= nown) break;
            sM[tid + r * CC_T] = acc[r];
            if (own_a[r] == own_b[r]) tr = cadd(tr, acc[r]);
        }
        __syncthreads();
        double2 ex = cmk(0.0, 0.0);
        if (g >= 0) {
#pragma unroll
            for (int r = 0; r < CC_OWN; ++r) {
                if (r >= nown) break;
                const int o = tid + r * CC_T, a = own_a[r], b = own_b[r];
                const int t = o < nu * nu ? b * nu + a : nu * nu + b * nd + a;
                cfma(ex, acc[r], sM[t]);
            }
        }
        const double2 v = cc_block_sum(tr, red);
        const double2 x = g >= 0 ? cc_block_sum(ex, red) : cmk(0.0, 0.0);
        if (tid == 0) {
            if (g < 0) {
                e_acc = cadd(e_acc, v);
            } else {
                vpair[pair * G + g] = v;
                const double2 v2 = cmul(v, v);
                e_acc.x += 0.5 * (v2.x - x.x);
                e_acc.y += 0.5 * (v2.y - x.y);
            }
        }
    }
    if (tid == 0) epair[pair] = e_acc;
}

static size_t contract_fp64c_smem(int N, int nu, int nd) {
    const size_t nt = nu + nd;
    return ((size_t)N * nu + (size_t)N * nt + (size_t)nu * CC_JB + (size_t)nu * nu + (size_t)nd * nd) * 16 +
           (size_t)N * CC_JB * 8;
}

bool contract_fp64c_supported(int N, int nu, int nd) {
    return nu * nu + nd * nd <= CC_OWN * CC_T && contract_fp64c_smem(N, nu, nd) <= 200 * 1024;
}

cudaError_t contract_fp64c(cudaStream_t s, const Dims& d, const double* h, const double* L, const double2* Phi,
                           const double2* Theta, double2* vpair, double2* epair, const int* list, const int* n_list) {
    if (!contract_fp64c_supported(d.N, d.nu, d.nd)) return cudaErrorInvalidValue;
    if (d.pairs <= 0) return cudaSuccess;
    const size_t smem = contract_fp64c_smem(d.N, d.nu, d.nd);
    cudaError_t e = raise_smem_limit((const void*)contract_fp64c_kernel, smem);
    if (e != cudaSuccess) return e;
    contract_fp64c_kernel<<<(unsigned)d.pairs, CC_T, smem, s>>>(d.N, d.nu, d.nd, d.G, h, L, Phi, Theta, vpair, epair,
                                                                 list, n_list);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace afq
