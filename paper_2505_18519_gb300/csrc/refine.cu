// Error-controlled refinement of the tensor-core contraction (mixed precision,
// per-pair form): the pairs that would put their walker's energy outside the
// tolerance are recomputed by the per-pair contraction kernel in double-float
// arithmetic (FP32 pairs, about 44 significant bits: some 2^24 times below the
// split-FP16 error, at FP32 instruction rates).
//
// The split-FP16 contraction carries about 20 significant bits per operand.
// Its local-energy error grows with the conditioning of the overlap: for pair p
// the typical error is close to
//   sigma_p = (2 / N) u Lambda ||Theta_p||_F^2,   u = 2^-20,   Lambda = sum_g ||L_g||_2^2,
// where ||Theta_p||_F = ||A_p^-1||_F for orthonormal walkers (Theta = phi A^-1).
// The errors of a walker's pairs are nearly independent, so the error of its
// sign-weighted average (Eq. (27)) is estimated as
//   eps_w = 2 sqrt(sum_p sigma_p^2) / |sum_p S_p|
// over the pairs whose tensor-core values it keeps.  Per walker, the pairs are
// taken in decreasing ||Theta_p||_F and recomputed until eps_w <= tol / 2,
// so the walker's error stays below tol.  The model and its constant 2 / N were
// fitted to the measured per-pair errors of systems with N = 50 .. 120.
#include "kernels.cuh"

namespace afq {

constexpr int RF_T = 256;
constexpr int RF_POWER_ITERS = 256;
constexpr int RF_MAXP = 1024;

// Sum over the block in a fixed order (warp shuffles, then warp 0); valid in
// every thread.
__device__ double rf_block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < RF_T / 32 ? red[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) red[RF_T / 32] = t;
    }
    __syncthreads();
    return red[RF_T / 32];
}

// ||L_g||_2^2 of the symmetric L_g by power iteration: ||L v_k||^2 with v_k
// the normalised iterate tends to the largest squared eigenvalue from below.
__global__ void __launch_bounds__(RF_T) chol_norm2_kernel(int N, const double* __restrict__ L, double* out) {
    extern __shared__ double sv[];   // 2N
    __shared__ double red[RF_T / 32 + 1];
    const double* Lg = L + blockIdx.x * (long long)N * N;
    double* v = sv;
    double* lv = sv + N;
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += RF_T) {
        v[i] = 1.0 + (double)i / N;
        s += v[i] * v[i];
    }
    s = rf_block_sum(s, red);
    const double inv0 = 1.0 / sqrt(s);
    for (int i = threadIdx.x; i < N; i += RF_T) v[i] *= inv0;
    double lam2 = 0.0;
    for (int it = 0; it < RF_POWER_ITERS; ++it) {
        __syncthreads();
        double part = 0.0;
        for (int i = threadIdx.x; i < N; i += RF_T) {
            double t = 0.0;
            for (int j = 0; j < N; ++j) t = fma(Lg[(long long)i * N + j], v[j], t);
            lv[i] = t;
            part += t * t;
        }
        lam2 = rf_block_sum(part, red);   // ||L v||^2 with ||v|| = 1
        if (!(lam2 > 0.0)) break;         // uniform across the block
        const double inv = 1.0 / sqrt(lam2);
        for (int i = threadIdx.x; i < N; i += RF_T) v[i] = lv[i] * inv;
    }
    if (threadIdx.x == 0) out[blockIdx.x] = lam2 > 0.0 ? lam2 : 0.0;
}

// Lambda = sum_g ||L_g||_2^2 in order g = 0 .. G-1.
__global__ void sum_in_order_kernel(int n, const double* __restrict__ x, double* out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += x[i];
        out[0] = s;
    }
}

cudaError_t refine_scale(cudaStream_t s, int N, int G, const double* L, double* lam_g, double* lam) {
    if (G <= 0) return cudaSuccess;
    const size_t smem = 2 * (size_t)N * sizeof(double);
    cudaError_t e = raise_smem_limit((const void*)chol_norm2_kernel, smem);
    if (e != cudaSuccess) return e;
    chol_norm2_kernel<<<G, RF_T, smem, s>>>(N, L, lam_g);
    sum_in_order_kernel<<<1, 32, 0, s>>>(G, lam_g, lam);
    count_launches(2);
    return cudaGetLastError();
}

// ||Theta_p||_F^2 over both spins, one warp per pair.
__global__ void __launch_bounds__(RF_T) theta_norm_kernel(int nn, long long pairs, const double2* __restrict__ Theta,
                                                          double* __restrict__ th2) {
    const long long pair = (long long)blockIdx.x * (RF_T / 32) + (threadIdx.x >> 5);
    if (pair >= pairs) return;
    const int lane = threadIdx.x & 31;
    const double2* T = Theta + pair * (long long)nn;
    double s = 0.0;
    for (int e = lane; e < nn; e += 32) {
        const double2 t = T[e];
        s = fma(t.x, t.x, fma(t.y, t.y, s));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) th2[pair] = s;
}

// One block per walker: sort the walker's pairs by ||Theta_p||_F^2 (bitonic,
// decreasing, ties by index), find how many of the largest must be refined, and
// append their indices to items (order of walkers in the list is arbitrary).
__global__ void __launch_bounds__(RF_T) refine_select_kernel(int N, int P, double tol, const double* __restrict__ lam,
                                                             const double2* __restrict__ logdet,
                                                             const double* __restrict__ th2, int spins, double u,
                                                             const int* __restrict__ alive, int* items, int* n_items,
                                                             unsigned long long* counters) {
    __shared__ double key[RF_MAXP];
    __shared__ int id[RF_MAXP];
    __shared__ double red[RF_T / 32 + 1];
    __shared__ int s_base, s_k;
    const long long w = blockIdx.x;
    if (alive && !alive[w]) return;
    int P2 = 1;
    while (P2 < P) P2 <<= 1;
    for (int i = threadIdx.x; i < P2; i += RF_T) {
        double k = -INFINITY;
        if (i < P) {
            k = spins ? th2[2 * (w * P + i)] + th2[2 * (w * P + i) + 1] : th2[w * P + i];
            if (!isfinite(k)) k = INFINITY;   // a singular or overflowing pair is always refined
        }
        key[i] = k;
        id[i] = i;
    }
    // sum_p S_p, S_p = exp(i Im log ov_p) (Eq. (26))
    double sx = 0.0, sy = 0.0;
    for (int p = threadIdx.x; p < P; p += RF_T) {
        const long long pair = w * P + p;
        double sn, cs;
        sincos(logdet[2 * pair].y + logdet[2 * pair + 1].y, &sn, &cs);
        sx += cs;
        sy += sn;
    }
    sx = rf_block_sum(sx, red);
    sy = rf_block_sum(sy, red);
    // bitonic sort into decreasing key (ties: lower index first)
    for (int size = 2; size <= P2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < P2; i += RF_T) {
                const int l = i ^ stride;
                if (l <= i) continue;
                const bool l_first = key[l] > key[i] || (key[l] == key[i] && id[l] < id[i]);
                const bool i_first = key[i] > key[l] || (key[i] == key[l] && id[i] < id[l]);
                if ((i & size) == 0 ? l_first : i_first) {
                    const double tk = key[i]; key[i] = key[l]; key[l] = tk;
                    const int ti = id[i]; id[i] = id[l]; id[l] = ti;
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double absS = sqrt(sx * sx + sy * sy);
        const double c = (2.0 / N) * u * lam[0];
        int k = P;   // pairs 0 .. k-1 (in sorted order) are refined
        if (absS > 0.0 && isfinite(absS)) {
            // keep the smallest pairs while their estimated error stays within tol / 2
            const double lim = 0.25 * tol * absS / c;   // 2 c sqrt(s2) / absS <= tol / 2
            double s2 = 0.0;
            for (int i = P - 1; i >= 0; --i) {
                const double t = key[i] * key[i];
                if (!(sqrt(s2 + t) <= lim)) break;
                s2 += t;
                k = i;
            }
        }
        s_k = k;
        s_base = k > 0 ? atomicAdd(n_items, k) : 0;
        if (k > 0) atomicAdd(&counters[5], (unsigned long long)k);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < s_k; i += RF_T) items[s_base + i] = (int)(w * P + id[i]);
}

cudaError_t refine_select(cudaStream_t s, const Dims& d, double tol, const double* lam, const double2* logdet,
                          const double2* Theta, double* th2, const int* alive, int* items, int* n_items,
                          unsigned long long* counters, const double* th2_spins, double u) {
    if (d.P > RF_MAXP) return cudaErrorInvalidValue;
    if (d.pairs <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(n_items, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const long long nb = (d.pairs + RF_T / 32 - 1) / (RF_T / 32);
    if (!th2_spins) {
        theta_norm_kernel<<<(unsigned)nb, RF_T, 0, s>>>(d.N * d.nt, d.pairs, Theta, th2);
        count_launches(1);
    }
    refine_select_kernel<<<d.W, RF_T, 0, s>>>(d.N, d.P, tol, lam, logdet, th2_spins ? th2_spins : th2, th2_spins ? 1 : 0,
                                              u, alive, items, n_items, counters);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace afq
