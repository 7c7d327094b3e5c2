// FP64 fused contraction of the local energy and force bias (the dominant work
// of a step).  For one pair (walker w, path p) with trial orbitals Phi (N x n_up,
// real) and Theta_s = phi_s (Phi_s^T phi_s)^-1 (N x n_s, complex) the mixed
// Green's function is G^s_ij = sum_a Theta_s,ja Phi_ia, so with
//   R_g = Phi^T L_g (n_up x N, real) and M_g,s = R_g[:n_s] Theta_s (n_s x n_s)
// the force-bias value is v_g = sum_s Tr M_g,s (Eq. (15), (27)) and the local
// energy (Eq. (1), (3), (16) by Wick's theorem) is
//   E_L = sum_s Tr(Phi_s^T h Theta_s) + 1/2 sum_g [ v_g^2 - sum_s Tr(M_g,s M_g,s) ].
// No matrix of the contraction goes to global memory: one block per pair keeps
// Phi and Theta in shared memory and streams column blocks of each L_g.
#include "kernels.cuh"

namespace afq {

constexpr int CT = 256;   // threads per block
constexpr int MAXOWN = 16;  // M entries owned per thread (n_up^2 + n_dn^2 <= 16 * 256)

__host__ __device__ __forceinline__ size_t r2(size_t x) { return (x + 1) & ~(size_t)1; }

__device__ __forceinline__ double2 block_sum2(double2 v, double2* red) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double2 t = cmk(0.0, 0.0);
    if (threadIdx.x < 32) {
        t = (lane < CT / 32) ? red[lane] : cmk(0.0, 0.0);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            t.x += __shfl_xor_sync(0xffffffffu, t.x, off);
            t.y += __shfl_xor_sync(0xffffffffu, t.y, off);
        }
    }
    __syncthreads();
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(CT) contract_fp64_kernel(int N, int nu, int nd, int G, int JB,
                                                           const double* __restrict__ h, const double* __restrict__ L,
                                                           const double* __restrict__ Phi, const double2* __restrict__ Theta,
                                                           double2* __restrict__ vpair, double2* __restrict__ epair) {
    extern __shared__ double smc[];
    __shared__ double2 red[CT / 32];
    const int nt = nu + nd;
    const long long pair = blockIdx.x;
    const size_t oTh = r2((size_t)N * nu), oL = oTh + 2 * (size_t)N * nt, oR = oL + (size_t)N * JB;
    const size_t oM = r2(oR + (size_t)nu * JB);
    double* sPhi = smc;                                             // N x nu
    double2* sTh = reinterpret_cast<double2*>(smc + oTh);           // N x nt
    double* sL = smc + oL;                                          // N x JB
    double* sR = smc + oR;                                          // nu x JB
    double2* sM = reinterpret_cast<double2*>(smc + oM);             // nu^2 + nd^2
    const int tid = threadIdx.x;
    const double* gPhi = Phi + pair * (long long)N * nu;
    const double2* gTh = Theta + pair * (long long)N * nt;
    for (int e = tid; e < N * nu; e += CT) sPhi[e] = gPhi[e];
    for (int e = tid; e < N * nt; e += CT) sTh[e] = gTh[e];
    const int nM = nu * nu + nd * nd;
    // decode owned M entries: o < nu^2 -> spin up (a, b); else spin down
    int own_a[MAXOWN], own_b[MAXOWN], own_c[MAXOWN];
    int nown = 0;
#pragma unroll
    for (int r = 0; r < MAXOWN; ++r) {
        int o = tid + r * CT;
        own_a[r] = own_b[r] = own_c[r] = 0;
        if (o >= nM) continue;
        nown = r + 1;
        if (o < nu * nu) { own_a[r] = o / nu; own_b[r] = o % nu; own_c[r] = o % nu; }
        else { int q = o - nu * nu; own_a[r] = q / nd; own_b[r] = q % nd; own_c[r] = nu + q % nd; }
    }
    double2 e_acc = cmk(0.0, 0.0);   // thread 0 accumulates E_L
    __syncthreads();
    for (int g = -1; g < G; ++g) {
        const double* Lg = (g < 0) ? h : L + (long long)g * N * N;
        double2 acc[MAXOWN];
#pragma unroll
        for (int r = 0; r < MAXOWN; ++r) acc[r] = cmk(0.0, 0.0);
        for (int j0 = 0; j0 < N; j0 += JB) {
            int jb = min(JB, N - j0);
            for (int e = tid; e < N * jb; e += CT) {
                int i = e / jb, j = e - i * jb;
                sL[i * JB + j] = Lg[(long long)i * N + j0 + j];
            }
            __syncthreads();
            for (int e = tid; e < nu * jb; e += CT) {
                int a = e / jb, j = e - a * jb;
                double s = 0.0;
                for (int i = 0; i < N; ++i) s = fma(sPhi[i * nu + a], sL[i * JB + j], s);
                sR[a * JB + j] = s;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < MAXOWN; ++r) {
                if (r >= nown) break;
                const double* Ra = sR + own_a[r] * JB;
                const double2* Tc = sTh + (size_t)j0 * nt + own_c[r];
                double2 s = acc[r];
                for (int j = 0; j < jb; ++j) {
                    double rv = Ra[j];
                    double2 t = Tc[(size_t)j * nt];
                    s.x = fma(rv, t.x, s.x);
                    s.y = fma(rv, t.y, s.y);
                }
                acc[r] = s;
            }
            __syncthreads();
        }
        // traces
        double2 tr = cmk(0.0, 0.0);
#pragma unroll
        for (int r = 0; r < MAXOWN; ++r) {
            if (r >= nown) break;
            int o = tid + r * CT;
            sM[o] = acc[r];
            if (own_a[r] == own_b[r]) tr = cadd(tr, acc[r]);
        }
        __syncthreads();
        double2 ex = cmk(0.0, 0.0);
        if (g >= 0) {
#pragma unroll
            for (int r = 0; r < MAXOWN; ++r) {
                if (r >= nown) break;
                int o = tid + r * CT;
                int a = own_a[r], b = own_b[r];
                int t = (o < nu * nu) ? (b * nu + a) : (nu * nu + b * nd + a);
                cfma(ex, acc[r], sM[t]);
            }
        }
        double2 v = block_sum2(tr, red);
        double2 x = (g >= 0) ? block_sum2(ex, red) : cmk(0.0, 0.0);
        if (tid == 0) {
            if (g < 0) {
                e_acc = cadd(e_acc, v);                  // one-body term sum_s Tr(Phi_s^T h Theta_s)
            } else {
                vpair[pair * G + g] = v;
                double2 v2 = cmul(v, v);
                e_acc.x += 0.5 * (v2.x - x.x);
                e_acc.y += 0.5 * (v2.y - x.y);
            }
        }
    }
    if (tid == 0) epair[pair] = e_acc;
}

size_t contract_fp64_smem(int N, int nu, int nd, int JB) {
    int nt = nu + nd;
    size_t oTh = r2((size_t)N * nu), oL = oTh + 2 * (size_t)N * nt, oR = oL + (size_t)N * JB;
    size_t oM = r2(oR + (size_t)nu * JB);
    return (oM + 2 * (size_t)(nu * nu + nd * nd)) * sizeof(double);
}

int contract_fp64_jb(int N) { return N <= 64 ? N : 32; }

bool contract_fp64_supported(int N, int nu, int nd) {
    if (nu * nu + nd * nd > MAXOWN * CT) return false;
    return contract_fp64_smem(N, nu, nd, contract_fp64_jb(N)) <= 220 * 1024;
}

cudaError_t contract_fp64(cudaStream_t s, const Dims& d, const double* h, const double* L, const double* Phi,
                          const double2* Theta, double2* vpair, double2* epair, long long pairs) {
    int JB = contract_fp64_jb(d.N);
    size_t smem = contract_fp64_smem(d.N, d.nu, d.nd, JB);
    if (!contract_fp64_supported(d.N, d.nu, d.nd)) return cudaErrorInvalidValue;
    cudaError_t e = raise_smem_limit((const void*)contract_fp64_kernel, smem);
    if (e != cudaSuccess) return e;
    contract_fp64_kernel<<<(unsigned)pairs, CT, smem, s>>>(d.N, d.nu, d.nd, d.G, JB, h, L, Phi, Theta, vpair, epair); count_launches(1);
    return cudaGetLastError();
}

}  // namespace afq
