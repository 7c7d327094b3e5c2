// Per-walker kernels of the leapfrog step (Sec. III A; Appendix B.2):
// path-sign averages (Eq. (25)-(27)), the mixed estimator (Eq. (16)), fields
// and force bias (Eq. (4), (15)), propagation B(x - xbar) (Eq. (5), (12)), the
// importance function (Eq. (14)), Metropolis proposals and acceptance of the
// paths (Eq. (23)), and the hand-off constraint (Eq. (17), (28)-(29)).
#include "df.cuh"
#include <algorithm>

#include "kernels.cuh"

namespace afq {

__device__ __forceinline__ uint32_t step_of(const unsigned long long* ctr) { return (uint32_t)ctr[0]; }

// ---------------------------------------------------------------- random draws
// out[r * cols + k] = normal number k of draw (tag, step, entity entity0 + r, sweep).
__global__ void fill_normals_kernel(double* out, long long rows, int cols, long long entity0, uint64_t seed, uint32_t tag,
                                    const unsigned long long* ctr, uint32_t sweep) {
    int blocks_per_row = (cols + 1) / 2;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * blocks_per_row) return;
    long long r = t / blocks_per_row;
    int j = (int)(t - r * blocks_per_row);
    double2 z = normal_pair(seed, tag, step_of(ctr), (uint32_t)(entity0 + r), sweep, (uint32_t)j);
    out[r * cols + 2 * j] = z.x;
    if (2 * j + 1 < cols) out[r * cols + 2 * j + 1] = z.y;
}

cudaError_t fill_normals(cudaStream_t s, double* out, long long rows, int cols, long long entity0, uint64_t seed,
                         uint32_t tag, const unsigned long long* ctr, uint32_t sweep) {
    long long n = rows * ((cols + 1) / 2);
    if (n <= 0) return cudaSuccess;
    fill_normals_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, rows, cols, entity0, seed, tag, ctr, sweep); count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- initial walkers
// phi_w = Phi(x_w) for both spins (spin down: first n_dn columns), as complex.
__global__ void walkers_from_trial_kernel(int N, int nu, int nd, const double* __restrict__ Phi_w, double2* phi) {
    long long w = blockIdx.x;
    int nt = nu + nd;
    for (int e = threadIdx.x; e < N * nt; e += blockDim.x) {
        int i = e / nt, c = e - i * nt;
        int src = c < nu ? c : c - nu;
        phi[w * (long long)N * nt + e] = cmk(Phi_w[w * (long long)N * nu + (long long)i * nu + src], 0.0);
    }
}

cudaError_t walkers_from_trial(cudaStream_t s, const Dims& d, const double* Phi_w, double2* phi) {
    walkers_from_trial_kernel<<<d.W, 128, 0, s>>>(d.N, d.nu, d.nd, Phi_w, phi); count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- block reductions
template <int NT>
__device__ __forceinline__ double2 bsum2(double2 v, double2* red) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < NT / 32) ? red[lane] : cmk(0.0, 0.0);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
        }
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    double2 r = red[0];
    __syncthreads();
    return r;   // every thread
}

// ---------------------------------------------------------------- path-sign averages
// logov_p = log det(up) + log det(down); S_p = exp(i Im logov_p) (Eq. (26));
// vbar_g = sum_p S_p v_pg / sum_p S_p and ebar = sum_p S_p E_p / sum_p S_p (Eq. (27)).
// The sums over p run in order p = 0..P-1 (deterministic).
__global__ void __launch_bounds__(256) walker_average_kernel(int P, int G, const double2* __restrict__ logdet,
                                                             const double2* __restrict__ vpair, const double2* __restrict__ epair,
                                                             double2* logov, double2* sumS_out, double2* vbar, double2* ebar) {
    extern __shared__ double2 sS[];   // P path signs
    long long w = blockIdx.x;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        long long pair = w * P + p;
        double2 lo = cadd(logdet[2 * pair], logdet[2 * pair + 1]);
        logov[pair] = lo;
        double s, c;
        sincos(lo.y, &s, &c);
        sS[p] = cmk(c, s);
    }
    __syncthreads();
    double2 sumS = cmk(0.0, 0.0), se = cmk(0.0, 0.0);
    for (int p = 0; p < P; ++p) {
        sumS = cadd(sumS, sS[p]);
        se = cadd(se, cmul(sS[p], epair[w * P + p]));
    }
    double2 inv = cdiv(cmk(1.0, 0.0), sumS);
    if (threadIdx.x == 0) {
        sumS_out[w] = sumS;
        ebar[w] = cmul(se, inv);
    }
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        double2 sv = cmk(0.0, 0.0);
        for (int p = 0; p < P; ++p) cfma(sv, sS[p], vpair[(w * P + p) * (long long)G + g]);
        vbar[w * (long long)G + g] = cmul(sv, inv);
    }
}

cudaError_t walker_average(cudaStream_t s, const Dims& d, const double2* logdet, const double2* vpair,
                           const double2* epair, double2* logov, double2* sumS, double2* vbar, double2* ebar) {
    cudaError_t e = raise_smem_limit((const void*)walker_average_kernel, d.P * sizeof(double2));
    if (e != cudaSuccess) return e;
    walker_average_kernel<<<d.W, 256, d.P * sizeof(double2), s>>>(d.P, d.G, logdet, vpair, epair, logov, sumS, vbar, ebar); count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- mixed estimator
// out3 = {sum_w W_w Re ebar_w, sum_w W_w, sum_w W_w |sum_p S_p| / P} over W_w > 0,
// one block, fixed-order tree reduction.
__global__ void __launch_bounds__(1024) energy_reduce_kernel(int W, int P, const double* __restrict__ weight,
                                                             const double2* __restrict__ ebar, const double2* __restrict__ sumS,
                                                             double* out3) {
    __shared__ double r0[1024], r1[1024], r2[1024];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        double wt = weight[w];
        // a walker without a finite estimate (non-finite orbitals) carries no weight
        if (wt > 0.0 && isfinite(ebar[w].x) && isfinite(ebar[w].y)) {
            a += wt * ebar[w].x;
            b += wt;
            c += wt * cabs_(sumS[w]) / P;
        }
    }
    r0[threadIdx.x] = a; r1[threadIdx.x] = b; r2[threadIdx.x] = c;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            r0[threadIdx.x] += r0[threadIdx.x + off];
            r1[threadIdx.x] += r1[threadIdx.x + off];
            r2[threadIdx.x] += r2[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out3[0] = r0[0]; out3[1] = r1[0]; out3[2] = r2[0]; }
}

cudaError_t energy_reduce(cudaStream_t s, const Dims& d, const double* weight, const double2* ebar,
                          const double2* sumS, double* out3) {
    energy_reduce_kernel<<<1, 1024, 0, s>>>(d.W, d.P, weight, ebar, sumS, out3); count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- fields and force bias
// Walkers with W = 0 or |sum_p S_p| <= threshold are dead (W = 0) and frozen.
// xi_g ~ N(0,1) (Philox, tag FIELD, entity w); xbar_g = -i sqrt(tau) vbar_g;
// y = xi - xbar written as planes (row 2w: Re y, row 2w+1: Im y);
// logshift = sum_g (xi_g xbar_g - xbar_g^2 / 2), the log of p(x - xbar)/p(x).
__global__ void __launch_bounds__(256) fields_kernel(int G, long long woff, uint64_t seed, double dtau, double thr,
                                                     const unsigned long long* ctr, const double2* __restrict__ vbar,
                                                     const double2* __restrict__ sumS, double* weight, int* alive,
                                                     double* yplanes, double2* logshift) {
    __shared__ double2 red[8];
    long long w = blockIdx.x;
    bool live = weight[w] > 0.0 && cabs_(sumS[w]) > thr;
    double* yre = yplanes + (2 * w) * (long long)G;
    double* yim = yre + G;
    if (!live) {
        for (int g = threadIdx.x; g < G; g += blockDim.x) { yre[g] = 0.0; yim[g] = 0.0; }
        if (threadIdx.x == 0) { weight[w] = 0.0; alive[w] = 0; logshift[w] = cmk(0.0, 0.0); }
        return;
    }
    uint32_t step = step_of(ctr);
    double st = sqrt(dtau);
    double2 acc = cmk(0.0, 0.0);
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        double xi = normal_at(seed, TAG_FIELD, step, (uint32_t)(woff + w), 0, (uint32_t)g);
        double2 v = vbar[w * (long long)G + g];
        double2 xb = cmk(st * v.y, -st * v.x);          // -i sqrt(tau) v
        yre[g] = xi - xb.x;
        yim[g] = -xb.y;
        double2 xb2 = cmul(xb, xb);
        acc.x += xi * xb.x - 0.5 * xb2.x;
        acc.y += xi * xb.y - 0.5 * xb2.y;
    }
    double2 tot = bsum2<256>(acc, red);
    if (threadIdx.x == 0) { alive[w] = 1; logshift[w] = tot; }
}

cudaError_t fields(cudaStream_t s, const Dims& d, const StepParams& p, const unsigned long long* ctr,
                   const double2* vbar, const double2* sumS, double* weight, int* alive, double* yplanes,
                   double2* logshift) {
    fields_kernel<<<d.W, 256, 0, s>>>(d.G, p.woff, p.seed, p.dtau, p.kill_threshold, ctr, vbar, sumS, weight, alive, yplanes,
                                      logshift); count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- propagation
// phi' = E (sum_{m<=order} A^m / m!) E phi with E = exp(-tau T/2) and
// A = i sqrt(tau) sum_g y_g L_g = -sqrt(tau) Q + i sqrt(tau) P, where
// P = sum_g Re(y_g) L_g, Q = sum_g Im(y_g) L_g (rows 2w, 2w+1 of Aplanes).
// One block per walker, both spins at once (N x nt complex); the running sum
// is kept in phi_new (global) and the current term in shared memory, or, when
// the two N x nt work arrays do not fit there (N = 200 with 40 + 40 electrons
// needs 512 KB), in the walker's slice of a global scratch buffer (L1/L2).
template <bool SMEM>
__global__ void __launch_bounds__(256) propagate_kernel(int N, int nt, int order, double dtau, const double* __restrict__ E,
                                                        const double* __restrict__ Aplanes, const double2* __restrict__ phi,
                                                        double2* phi_new, const int* __restrict__ alive,
                                                        double2* scratch) {
    extern __shared__ double2 sv[];
    long long w = blockIdx.x;
    double2* work = SMEM ? sv : scratch + w * 2 * (long long)N * nt;
    double2* V = work;                     // N x nt
    double2* Wt = work + (size_t)N * nt;   // N x nt
    const double2* in = phi + w * (long long)N * nt;
    double2* acc = phi_new + w * (long long)N * nt;
    int nn = N * nt;
    if (!alive[w]) {
        for (int e = threadIdx.x; e < nn; e += blockDim.x) acc[e] = in[e];
        return;
    }
    const double* Pm = Aplanes + (2 * w) * (long long)N * N;
    const double* Qm = Pm + (long long)N * N;
    double st = sqrt(dtau);
    for (int e = threadIdx.x; e < nn; e += blockDim.x) V[e] = in[e];
    __syncthreads();
    // V <- E V ; acc <- V
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        int i = e / nt, c = e - i * nt;
        double2 s = cmk(0.0, 0.0);
        for (int j = 0; j < N; ++j) {
            double ev = E[(long long)i * N + j];
            double2 v = V[j * nt + c];
            s.x = fma(ev, v.x, s.x);
            s.y = fma(ev, v.y, s.y);
        }
        Wt[e] = s;
        acc[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) V[e] = Wt[e];
    __syncthreads();
    for (int m = 1; m <= order; ++m) {
        double inv = 1.0 / m;
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            int i = e / nt, c = e - i * nt;
            double pr = 0.0, pi = 0.0, qr = 0.0, qi = 0.0;   // (P V), (Q V)
            for (int j = 0; j < N; ++j) {
                double pv = Pm[(long long)i * N + j], qv = Qm[(long long)i * N + j];
                double2 v = V[j * nt + c];
                pr = fma(pv, v.x, pr); pi = fma(pv, v.y, pi);
                qr = fma(qv, v.x, qr); qi = fma(qv, v.y, qi);
            }
            // A V = (-st Q + i st P) V
            double2 t = cmk(st * (-qr - pi) * inv, st * (-qi + pr) * inv);
            Wt[e] = t;
            acc[e] = cadd(acc[e], t);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nn; e += blockDim.x) V[e] = Wt[e];
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nn; e += blockDim.x) V[e] = acc[e];
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        int i = e / nt, c = e - i * nt;
        double2 s = cmk(0.0, 0.0);
        for (int j = 0; j < N; ++j) {
            double ev = E[(long long)i * N + j];
            double2 v = V[j * nt + c];
            s.x = fma(ev, v.x, s.x);
            s.y = fma(ev, v.y, s.y);
        }
        acc[e] = s;
    }
}

bool propagate_in_smem(int N, int nt) { return 2 * (size_t)N * nt * 16 <= 220 * 1024; }

cudaError_t propagate(cudaStream_t s, const Dims& d, const StepParams& p, const double* expT, const double* Aplanes,
                      const double2* phi, double2* phi_new, const int* alive, double2* scratch) {
    if (propagate_in_smem(d.N, d.nt)) {
        const size_t smem = 2 * (size_t)d.N * d.nt * sizeof(double2);
        cudaError_t e = raise_smem_limit((const void*)propagate_kernel<true>, smem);
        if (e != cudaSuccess) return e;
        propagate_kernel<true><<<d.W, 256, smem, s>>>(d.N, d.nt, p.taylor_order, p.dtau, expT, Aplanes, phi, phi_new,
                                                      alive, nullptr);
    } else {
        if (!scratch) return cudaErrorInvalidValue;
        propagate_kernel<false><<<d.W, 256, 0, s>>>(d.N, d.nt, p.taylor_order, p.dtau, expT, Aplanes, phi, phi_new,
                                                    alive, scratch);
    }
    count_launches(1);
    return cudaGetLastError();
}

// Mixed-precision form of the same propagation (Eq. (12)): E and the planes
// P, Q arrive as double-float pairs, the vectors V are held as double-float in
// shared memory, every matrix-vector product is a Dot2 sum, and the series
// acc = sum_m (A^m / m!) E phi is summed in FP64.  FP32 instructions issue at
// 64 times the FP64 rate here, and the double-float products carry about 44
// significant bits, far below the tensor-core contraction's error.
__device__ __forceinline__ float4 df_pack(dfl re, dfl im) { return make_float4(re.hi, re.lo, im.hi, im.lo); }

__global__ void __launch_bounds__(256) propagate_df_kernel(int N, int nt, int order, double dtau,
                                                           const dfl* __restrict__ E, const dfl* __restrict__ Aplanes,
                                                           const double2* __restrict__ phi, double2* phi_new,
                                                           const int* __restrict__ alive) {
    extern __shared__ float4 sdf[];
    float4* V = sdf;                          // N x nt, (Re hi, Re lo, Im hi, Im lo)
    float4* Wt = sdf + (size_t)N * nt;        // N x nt
    const long long w = blockIdx.x;
    const double2* in = phi + w * (long long)N * nt;
    double2* acc = phi_new + w * (long long)N * nt;
    const int nn = N * nt;
    if (!alive[w]) {
        for (int e = threadIdx.x; e < nn; e += blockDim.x) acc[e] = in[e];
        return;
    }
    const dfl* Pm = Aplanes + (2 * w) * (long long)N * N;
    const dfl* Qm = Pm + (long long)N * N;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        const double2 v = in[e];
        V[e] = df_pack(df_from(v.x), df_from(v.y));
    }
    __syncthreads();
    // Every product below: a thread takes row i and the four columns c = cg + k NG
    // (k < 4, NG = ceil(nt / 4); consecutive threads, consecutive columns), so that each
    // load of a matrix entry serves four sums; every sum runs over j in order as before.
    const int NG = (nt + 3) / 4;
    // acc <- E phi
    for (int it = threadIdx.x; it < N * NG; it += blockDim.x) {
        const int i = it / NG, cg = it - i * NG;
        float rh[4], rl[4], ih[4], il[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) rh[k] = rl[k] = ih[k] = il[k] = 0.f;
        for (int j = 0; j < N; ++j) {
            const dfl ev = E[(long long)i * N + j];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = min(cg + k * NG, nt - 1);
                const float4 v = V[j * nt + c];
                dot2_fma(rh[k], rl[k], ev, dfl{v.x, v.y});
                dot2_fma(ih[k], il[k], ev, dfl{v.z, v.w});
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = cg + k * NG;
            if (c >= nt) continue;
            const dfl re = df_two_sum(rh[k], rl[k]), im = df_two_sum(ih[k], il[k]);
            Wt[i * nt + c] = df_pack(re, im);
            acc[i * nt + c] = make_double2(df_to(re), df_to(im));
        }
    }
    __syncthreads();
    float4* cur = Wt;
    float4* nxt = V;
    const double st = sqrt(dtau);
    for (int m = 1; m <= order; ++m) {
        const dfl scale = df_from(st / m);
        for (int it = threadIdx.x; it < N * NG; it += blockDim.x) {
            const int i = it / NG, cg = it - i * NG;
            // A V = (-st Q + i st P) V: Re = -(Q Re V) - (P Im V), Im = (P Re V) - (Q Im V)
            float rh[4], rl[4], ih[4], il[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) rh[k] = rl[k] = ih[k] = il[k] = 0.f;
            for (int j = 0; j < N; ++j) {
                const dfl pv = Pm[(long long)i * N + j], qv = Qm[(long long)i * N + j];
                const dfl npv = df_neg(pv), nqv = df_neg(qv);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int c = min(cg + k * NG, nt - 1);
                    const float4 v = cur[j * nt + c];
                    const dfl vr{v.x, v.y}, vi{v.z, v.w};
                    dot2_fma(rh[k], rl[k], nqv, vr);
                    dot2_fma(rh[k], rl[k], npv, vi);
                    dot2_fma(ih[k], il[k], pv, vr);
                    dot2_fma(ih[k], il[k], nqv, vi);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = cg + k * NG;
                if (c >= nt) continue;
                const dfl re = df_mul(df_two_sum(rh[k], rl[k]), scale), im = df_mul(df_two_sum(ih[k], il[k]), scale);
                nxt[i * nt + c] = df_pack(re, im);
                const double2 a = acc[i * nt + c];
                acc[i * nt + c] = make_double2(a.x + df_to(re), a.y + df_to(im));
            }
        }
        __syncthreads();   // every read of cur is done before it is overwritten as nxt
        float4* t = cur; cur = nxt; nxt = t;
    }
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        const double2 a = acc[e];
        V[e] = df_pack(df_from(a.x), df_from(a.y));
    }
    __syncthreads();
    // phi' <- E acc
    for (int it = threadIdx.x; it < N * NG; it += blockDim.x) {
        const int i = it / NG, cg = it - i * NG;
        float rh[4], rl[4], ih[4], il[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) rh[k] = rl[k] = ih[k] = il[k] = 0.f;
        for (int j = 0; j < N; ++j) {
            const dfl ev = E[(long long)i * N + j];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = min(cg + k * NG, nt - 1);
                const float4 v = V[j * nt + c];
                dot2_fma(rh[k], rl[k], ev, dfl{v.x, v.y});
                dot2_fma(ih[k], il[k], ev, dfl{v.z, v.w});
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = cg + k * NG;
            if (c >= nt) continue;
            acc[i * nt + c] = make_double2(df_to(df_two_sum(rh[k], rl[k])), df_to(df_two_sum(ih[k], il[k])));
        }
    }
}

cudaError_t propagate_df(cudaStream_t s, const Dims& d, const StepParams& p, const void* expTdf, const void* Aplanes_df,
                         const double2* phi, double2* phi_new, const int* alive) {
    size_t smem = 2 * (size_t)d.N * d.nt * sizeof(float4);
    if (!propagate_in_smem(d.N, d.nt)) return cudaErrorInvalidValue;
    cudaError_t e = raise_smem_limit((const void*)propagate_df_kernel, smem);
    if (e != cudaSuccess) return e;
    propagate_df_kernel<<<d.W, 256, smem, s>>>(d.N, d.nt, p.taylor_order, p.dtau, reinterpret_cast<const dfl*>(expTdf),
                                               reinterpret_cast<const dfl*>(Aplanes_df), phi, phi_new, alive);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- overlap ratio and importance function
// For live walkers: logov'_p at phi' of the current paths; the sampled-trial
// ratio (Eq. (25)) = sum_p S_p exp(logov'_p - logov_p) / sum_p S_p, and
// |I| = |exp(logshift) * ratio| (Eq. (14)).
__global__ void __launch_bounds__(128) ratios_walker_kernel(int P, const double2* __restrict__ logov,
                                                            const double2* __restrict__ logdet_new,
                                                            const double2* __restrict__ sumS,
                                                            const double2* __restrict__ logshift,
                                                            const int* __restrict__ alive, double2* logov_cur,
                                                            double2* old_sum, double2* ratio, double* Iabs) {
    long long w = blockIdx.x;
    if (!alive[w]) return;
    __shared__ double2 terms[1024];
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        long long pair = w * P + p;
        double2 lo = logov[pair];
        double2 ln = cadd(logdet_new[2 * pair], logdet_new[2 * pair + 1]);
        logov_cur[pair] = ln;
        double s, c;
        sincos(lo.y, &s, &c);
        terms[p] = cmul(cmk(c, s), cexp_(csub(ln, lo)));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 os = cmk(0.0, 0.0);
        for (int p = 0; p < P; ++p) os = cadd(os, terms[p]);
        double2 r = cdiv(os, sumS[w]);
        old_sum[w] = os;
        ratio[w] = r;
        double2 I = cmul(cexp_(logshift[w]), r);
        Iabs[w] = cabs_(I);
    }
}

cudaError_t ratios(cudaStream_t s, const Dims& d, const double2* logov, const double2* logdet_new,
                   const double2* sumS, const double2* logshift, const int* alive, double2* logov_cur,
                   double2* old_sum, double2* ratio, double* Iabs) {
    if (d.P > 1024) return cudaErrorInvalidValue;
    ratios_walker_kernel<<<d.W, 128, 0, s>>>(d.P, logov, logdet_new, sumS, logshift, alive, logov_cur, old_sum, ratio,
                                             Iabs); count_launches(1);
    return cudaGetLastError();
}

// logov = sum over spins of logdet (used at init, before the burn-in sweeps).
__global__ void combine_logdet_kernel(long long pairs, const double2* __restrict__ logdet, double2* logov) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < pairs) logov[p] = cadd(logdet[2 * p], logdet[2 * p + 1]);
}

cudaError_t combine_logdet(cudaStream_t s, long long pairs, const double2* logdet, double2* logov) {
    combine_logdet_kernel<<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(pairs, logdet, logov); count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Metropolis on the paths
// Proposal for pair q (xi ~ N(0, I): Philox, tag PROPOSE or BURN_PROPOSE,
// entity q, this sweep):
//   prior  x' = xi                       pCN  x' = sqrt(1 - beta^2) x + beta xi
//   RW     x' = x + s xi                 MLP  x' = mu_w + exp(logv_w / 2) xi, or, with
//   probability mix (second uniform of the pair's ACCEPT draw), the RW move.
__device__ __forceinline__ bool mlp_uses_rw(uint64_t seed, uint32_t tag_acc, uint32_t step, uint32_t entity,
                                            uint32_t sweep, double mix) {
    Philox4 b = stream_block(seed, tag_acc, step, entity, sweep, 0);
    return u53(b.w[2], b.w[3]) < mix;
}

__global__ void propose_kernel(long long pairs, int P, int K, long long woff, uint64_t seed, uint32_t tag, uint32_t tag_acc,
                               uint32_t sweep, const unsigned long long* ctr, int proposal, double beta, double rw_step,
                               double mix, const double* __restrict__ x, const int* __restrict__ alive,
                               const float* __restrict__ mu, const float* __restrict__ logv, double* xprop) {
    int bpr = (K + 1) / 2;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pairs * bpr) return;
    long long q = t / bpr;
    int j = (int)(t - q * bpr);
    double* out = xprop + q * K;
    if (!alive[q / P]) {
        out[2 * j] = 0.0;
        if (2 * j + 1 < K) out[2 * j + 1] = 0.0;
        return;
    }
    const uint32_t step = step_of(ctr), ent = (uint32_t)(woff * P + q);
    double2 z = normal_pair(seed, tag, step, ent, sweep, (uint32_t)j);
    const double* xo = x + q * K;
    const int k0 = 2 * j, k1 = 2 * j + 1;
    bool rw = proposal == AFQMC_PROPOSAL_RW ||
              (proposal == AFQMC_PROPOSAL_MLP && mlp_uses_rw(seed, tag_acc, step, ent, sweep, mix));
    double v0, v1 = 0.0;
    if (proposal == AFQMC_PROPOSAL_PCN) {
        double a = sqrt(1.0 - beta * beta);
        v0 = fma(a, xo[k0], beta * z.x);
        if (k1 < K) v1 = fma(a, xo[k1], beta * z.y);
    } else if (rw) {
        v0 = fma(rw_step, z.x, xo[k0]);
        if (k1 < K) v1 = fma(rw_step, z.y, xo[k1]);
    } else if (proposal == AFQMC_PROPOSAL_MLP) {
        const long long w = q / P;
        v0 = fma(exp(0.5 * (double)logv[w * K + k0]), z.x, (double)mu[w * K + k0]);
        if (k1 < K) v1 = fma(exp(0.5 * (double)logv[w * K + k1]), z.y, (double)mu[w * K + k1]);
    } else {
        v0 = z.x;
        v1 = z.y;
    }
    out[k0] = v0;
    if (k1 < K) out[k1] = v1;
}

cudaError_t propose(cudaStream_t s, const Dims& d, const StepParams& p, const unsigned long long* ctr, uint32_t tag,
                    uint32_t tag_acc, uint32_t sweep, const double* x, const int* alive, const float* mu,
                    const float* logv, double* xprop) {
    long long n = d.pairs * ((d.K + 1) / 2);
    propose_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d.pairs, d.P, d.K, p.woff, p.seed, tag, tag_acc, sweep, ctr,
                                                               p.proposal, p.pcn_beta, p.rw_step, p.mlp_mix, x, alive, mu,
                                                               logv, xprop); count_launches(1);
    return cudaGetLastError();
}

// Metropolis-Hastings: log alpha = Re(logov'' - logov') + extra with
//   prior, pCN: extra = 0 (the prior is the proposal's invariant law)
//   RW:         extra = -(|x'|^2 - |x|^2) / 2
//   MLP move:   extra = -(|x'|^2 - |x|^2) / 2 + sum_k [(x'-mu)^2 - (x-mu)^2] / (2 v)
// accept iff log alpha >= 0 or u < exp(log alpha), u the first 53-bit uniform of
// (tag, step, pair, sweep); on acceptance copy x', Phi(x') and logov''.
// One block per pair.
__global__ void __launch_bounds__(128) accept_kernel(int N, int nu, int K, int P, long long woff, uint64_t seed, uint32_t tag,
                                                     uint32_t sweep, const unsigned long long* ctr, int proposal,
                                                     double mix, const double2* __restrict__ logdet_prop,
                                                     const double* __restrict__ xprop, const double* __restrict__ Phiprop,
                                                     const int* __restrict__ alive, const float* __restrict__ mu,
                                                     const float* __restrict__ logv, double2* logov_cur, double* x,
                                                     double* Phi, unsigned long long* counters, int* rdirty) {
    long long q = blockIdx.x;
    if (!alive[q / P]) return;
    __shared__ int acc;
    if (threadIdx.x == 0) {
        const uint32_t step = step_of(ctr), ent = (uint32_t)(woff * P + q);
        double2 ln = cadd(logdet_prop[2 * q], logdet_prop[2 * q + 1]);
        double delta = ln.x - logov_cur[q].x;
        if (proposal == AFQMC_PROPOSAL_RW || proposal == AFQMC_PROPOSAL_MLP) {
            const double* xo = x + q * K;
            const double* xn = xprop + q * K;
            double e = 0.0;
            for (int k = 0; k < K; ++k) e += xn[k] * xn[k] - xo[k] * xo[k];
            delta -= 0.5 * e;
            if (proposal == AFQMC_PROPOSAL_MLP && !mlp_uses_rw(seed, tag, step, ent, sweep, mix)) {
                const long long w = q / P;
                double g = 0.0;
                for (int k = 0; k < K; ++k) {
                    double m = mu[w * K + k], iv = exp(-(double)logv[w * K + k]);
                    double rn = xn[k] - m, ro = xo[k] - m;
                    g += (rn * rn - ro * ro) * iv;
                }
                delta += 0.5 * g;
            }
        }
        double u = uniform_at0(seed, tag, step, ent, sweep);
        int a = (delta >= 0.0) || (u < exp(delta));
        acc = a;
        if (a) {
            logov_cur[q] = ln;
            atomicAdd(&counters[3], 1ull);
            if (rdirty) rdirty[q] = 1;   // the pair's cached half-rotated matrices are stale
        }
        atomicAdd(&counters[4], 1ull);
    }
    __syncthreads();
    if (!acc) return;
    for (int k = threadIdx.x; k < K; k += blockDim.x) x[q * K + k] = xprop[q * K + k];
    long long nn = (long long)N * nu;
    for (long long e = threadIdx.x; e < nn; e += blockDim.x) Phi[q * nn + e] = Phiprop[q * nn + e];
}

cudaError_t accept(cudaStream_t s, const Dims& d, const StepParams& p, const unsigned long long* ctr, uint32_t tag,
                   uint32_t sweep, const double2* logdet_prop, const double* xprop, const double* Phiprop,
                   const int* alive, const float* mu, const float* logv, double2* logov_cur, double* x, double* Phi,
                   unsigned long long* counters, int* rdirty) {
    // the kernel copies N x nu doubles of an accepted pair's Phi: complex orbitals take twice as many
    accept_kernel<<<(unsigned)d.pairs, 128, 0, s>>>(d.N, d.cphi ? 2 * d.nu : d.nu, d.K, d.P, p.woff, p.seed, tag, sweep, ctr, p.proposal,
                                                    p.mlp_mix, logdet_prop, xprop, Phiprop, alive, mu, logv, logov_cur, x,
                                                    Phi, counters, rdirty); count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- hand-off constraint
// dtheta = Arg ratio; dtheta_T = Arg sum_p S'_p - Arg old_sum (Eq. (28)), then
// combined:   W *= |I| max(0, cos(dtheta + dtheta_T))
// separate:   W *= |I| max(0, cos dtheta) max(0, cos dtheta_T)
// half-plane: W *= |I| max(0, cos dtheta) [|wrap(dtheta_T)| <= pi/2]
// and W *= exp(tau E_T).  Non-finite weights become 0.  One warp per walker.
__global__ void handoff_kernel(int W, int P, int constraint, int importance, double dtau, double e_shift,
                               const double2* __restrict__ logov_cur, const double2* __restrict__ old_sum,
                               const double2* __restrict__ ratio, const double* __restrict__ Iabs,
                               const double2* __restrict__ ebar, const int* __restrict__ alive, double* weight,
                               int* status) {
    long long w = blockIdx.x;
    if (!alive[w]) return;
    int lane = threadIdx.x;
    // fixed-order sum over paths: lane 0 adds sequentially for bitwise determinism
    if (lane != 0) return;
    double2 ns = cmk(0.0, 0.0);
    for (int p = 0; p < P; ++p) {
        double s, c;
        sincos(logov_cur[w * P + p].y, &s, &c);
        ns = cadd(ns, cmk(c, s));
    }
    double dth = atan2(ratio[w].y, ratio[w].x);
    double dthT = atan2(ns.y, ns.x) - atan2(old_sum[w].y, old_sum[w].x);
    double f;
    if (constraint == AFQMC_CONSTRAINT_COMBINED) {
        f = fmax(0.0, cos(dth + dthT));
    } else if (constraint == AFQMC_CONSTRAINT_SEPARATE) {
        f = fmax(0.0, cos(dth)) * fmax(0.0, cos(dthT));
    } else {
        double wr = atan2(sin(dthT), cos(dthT));
        f = fmax(0.0, cos(dth)) * (fabs(wr) <= 0.5 * M_PI ? 1.0 : 0.0);
    }
    // |I|: hybrid form (Eq. (14) with the ratio of Eq. (25)), or the local-energy
    // form exp(-tau Re E_w) with E_w of Eq. (27) at the start of the step (Sec. III A)
    const double ia = importance == AFQMC_IMPORTANCE_LOCAL_ENERGY ? exp(-dtau * ebar[w].x) : Iabs[w];
    double wn = weight[w] * ia * f * exp(dtau * e_shift);
    if (!isfinite(wn)) {
        wn = 0.0;
        atomicOr(status, STATUS_NONFINITE);
    }
    weight[w] = wn;
}

cudaError_t handoff(cudaStream_t s, const Dims& d, const StepParams& p, const double2* logov_cur,
                    const double2* old_sum, const double2* ratio, const double* Iabs, const double2* ebar,
                    const int* alive, double* weight, int* status) {
    handoff_kernel<<<d.W, 32, 0, s>>>(d.W, d.P, p.constraint, p.importance, p.dtau, p.e_shift, logov_cur, old_sum,
                                      ratio, Iabs, ebar, alive, weight, status); count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- population control
// Comb (branching random walk, Sec. II B and II D; the scheme is this code's
// reading): after every `period`-th step the W weights are laid end to end on
// [0, sum W), W teeth spaced sum W / W apart starting at u sum W / W each pick
// the walker whose interval holds them (walker w gets c_w copies), and every
// new walker gets weight sum W / W.  A walker with c_w >= 1 keeps its slot; the
// extra copies, in increasing walker order, fill the slots of the walkers with
// c_w = 0, in increasing order, so the state is gathered in place and only the
// replaced slots move.  u is one Philox uniform (tag COMB, entity = global index
// of walker 0, the step's index).  Whether a step combs is decided here from the
// device step counter, so the same launches serve every step of a captured
// graph; the gather does nothing on the other steps.
constexpr int COMB_T = 1024;
constexpr int COMB_STAGE = 4096;    // weights staged in shared memory per pass of the running sum
constexpr int COMB_CHUNK = 2048;    // doubles per work item of the gather

// Exclusive prefix sum of one int per thread over the block; *total gets the sum.
__device__ int comb_block_scan(int v, int* sh, int* total) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < COMB_T; off <<= 1) {
        const int t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    const int incl = sh[threadIdx.x];
    *total = sh[COMB_T - 1];
    __syncthreads();
    return incl - v;
}

// One block.  Writes flag[0] (whether this step combs), flag[1] (replaced
// walkers n), slot[0..n) the replaced slots in increasing order and from[0..n)
// the walker each one copies.
__global__ void __launch_bounds__(COMB_T) comb_select_kernel(int W, int period, uint64_t seed, uint32_t entity,
                                                             unsigned long long* counters, double* weight,
                                                             double* cum, int* hit, int* slot, int* from,
                                                             int* flag) {
    __shared__ double s_w[COMB_STAGE];
    __shared__ double s_width, s_u, s_acc;
    __shared__ int s_last, s_do;
    __shared__ int sh[COMB_T];
    if (threadIdx.x == 0) {
        const unsigned long long done = counters[0];   // steps taken, this one included
        s_do = period > 0 && done > 0 && done % (unsigned long long)period == 0;
        s_u = s_do ? uniform_at0(seed, TAG_COMB, (uint32_t)(done - 1), entity, 0) : 0.0;
        s_acc = 0.0;
        s_last = -1;
    }
    __syncthreads();
    if (!s_do) {
        if (threadIdx.x == 0) flag[0] = 0;
        return;
    }
    // running sum, left to right, by one thread over weights staged in shared memory
    for (int base = 0; base < W; base += COMB_STAGE) {
        const int n = min(COMB_STAGE, W - base);
        for (int i = threadIdx.x; i < n; i += COMB_T) s_w[i] = weight[base + i];
        __syncthreads();
        if (threadIdx.x == 0) {
            double acc = s_acc;
            int last = s_last;
            for (int i = 0; i < n; ++i) {
                const double x = s_w[i];
                if (x > 0.0) last = base + i;
                acc += x;
                cum[base + i] = acc;
            }
            s_acc = acc;
            s_last = last;
        }
        __syncthreads();
    }
    const double total = s_acc;
    if (!(total > 0.0 && isfinite(total)) || s_last < 0) {   // nothing to resample from (uniform)
        if (threadIdx.x == 0) flag[0] = 0;
        return;
    }
    const double width = total / W, u = s_u;
    // tooth j -> walker (nondecreasing in j), kept in `slot` until the ranking below
    // has read it; `hit` marks the walkers some tooth picked
    for (int j = threadIdx.x; j < W; j += COMB_T) {
        const double pos = ((double)j + u) * width;
        int lo = 0, hi = W;   // first w with cum[w] > pos, W if none
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cum[mid] > pos) hi = mid; else lo = mid + 1;
        }
        slot[j] = min(lo, s_last);
        hit[j] = 0;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < W; j += COMB_T) hit[slot[j]] = 1;   // same value from every writer
    __syncthreads();
    // each thread takes a contiguous range of indices; free slots (walkers not hit)
    // and extra teeth (a tooth on the same walker as the one before) are ranked in
    // increasing index order by block scans
    const int per = (W + COMB_T - 1) / COMB_T;
    const int j0 = min(W, (int)threadIdx.x * per), j1 = min(W, j0 + per);
    int n_free = 0, n_extra = 0;
    for (int j = j0; j < j1; ++j) {
        n_free += hit[j] == 0;
        n_extra += j > 0 && slot[j] == slot[j - 1];
    }
    int total_free, total_extra;
    int r_free = comb_block_scan(n_free, sh, &total_free);
    int r_extra = comb_block_scan(n_extra, sh, &total_extra);
    for (int j = j0; j < j1; ++j)
        if (j > 0 && slot[j] == slot[j - 1]) from[r_extra++] = slot[j];
    __syncthreads();   // every tooth was read; `slot` now takes the replaced slots
    for (int j = j0; j < j1; ++j)
        if (!hit[j]) slot[r_free++] = j;
    for (int j = threadIdx.x; j < W; j += COMB_T) weight[j] = width;   // every read of weight came before
    if (threadIdx.x == 0) {
        flag[0] = 1;
        flag[1] = total_free;
        counters[6] += 1;
        counters[7] += (unsigned long long)total_free;
    }
}

// The walker-state arrays, rows of len[b] doubles per walker (a[3]: the cached
// half-rotated matrices, len[3] = 0 without them), and the per-walker rows of
// flen ints of their dirty flags (nullable).
struct CombRows {
    double* a[4];
    long long len[4];
    int* flags;
    int flen;
};

// Replaced slot slot[r] of every state array gets the row of walker from[r];
// those sources keep their own slots, so the copy is in place.  Work items are
// chunks of COMB_CHUNK doubles of one row of one array; the item that copies the
// first chunk of a slot's phi also copies its flags.
__global__ void __launch_bounds__(256) comb_gather_kernel(CombRows r, const int* __restrict__ slot,
                                                          const int* __restrict__ from, const int* __restrict__ flag) {
    if (!flag[0]) return;
    const long long n = flag[1];
    long long c[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) c[b] = (r.len[b] + COMB_CHUNK - 1) / COMB_CHUNK;
    const long long per_slot = c[0] + c[1] + c[2] + c[3];
    for (long long it = blockIdx.x; it < n * per_slot; it += gridDim.x) {
        const long long q = it / per_slot;
        long long k = it - q * per_slot;
        int b = 0;
        if (k >= c[0]) {
            k -= c[0]; b = 1;
            if (k >= c[1]) {
                k -= c[1]; b = 2;
                if (k >= c[2]) { k -= c[2]; b = 3; }
            }
        }
        const long long len = b == 0 ? r.len[0] : b == 1 ? r.len[1] : b == 2 ? r.len[2] : r.len[3];
        double* base = b == 0 ? r.a[0] : b == 1 ? r.a[1] : b == 2 ? r.a[2] : r.a[3];
        const long long src = from[q], dst = slot[q];
        const double* in = base + src * len;
        double* o = base + dst * len;
        const long long e1 = min(len, (k + 1) * COMB_CHUNK);
        for (long long e = k * COMB_CHUNK + threadIdx.x; e < e1; e += 256) o[e] = in[e];
        if (b == 0 && k == 0 && r.flags)
            for (int e = threadIdx.x; e < r.flen; e += 256) r.flags[dst * r.flen + e] = r.flags[src * r.flen + e];
    }
}

cudaError_t population_control(cudaStream_t s, const Dims& d, const StepParams& p, unsigned long long* counters,
                               double* weight, double2* phi, double* x, double* Phi, double* Rc, int* rdirty,
                               double* cum, int* hit, int* slot, int* from, int* flag) {
    if (p.pop_period <= 0) return cudaSuccess;
    comb_select_kernel<<<1, COMB_T, 0, s>>>(d.W, p.pop_period, p.seed, (uint32_t)p.woff, counters, weight, cum, hit,
                                            slot, from, flag);
    const long long rlen = Rc ? (long long)d.P * (d.G + 1) * d.N * d.nu : 0;
    CombRows rows{{(double*)phi, x, Phi, Rc},
                  {(long long)d.N * d.nt * 2, (long long)d.P * d.K, (long long)d.P * phi_stride(d), rlen},
                  Rc ? rdirty : nullptr, d.P};
    comb_gather_kernel<<<2 * 152, 256, 0, s>>>(rows, slot, from, flag);
    count_launches(2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- extra measurement paths
// Measurement-only paths (Sec. III A, last paragraph; Appendix B.3): the walkers
// that count (W > 0, |sum_p S_p| above the kill threshold at the propagation's
// paths), the sums over every round's paths, and the estimate with the factor
// R_w = (sum' S' / P') / (sum S / P) in numerator and denominator.
__global__ void meas_alive_kernel(int W, double thr, const double* __restrict__ weight,
                                  const double2* __restrict__ sumS, int* alive) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < W) alive[w] = weight[w] > 0.0 && cabs_(sumS[w]) > thr;
}

// acc[2w] += sum_p S_p E_L,p and acc[2w + 1] += sum_p S_p (in path order), S_p = exp(i Im log ov_p).
__global__ void meas_accumulate_kernel(int W, int P, const double2* __restrict__ logov,
                                       const double2* __restrict__ epair, const int* __restrict__ alive,
                                       double2* acc) {
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W || !alive[w]) return;
    double2 num = acc[2 * w], den = acc[2 * w + 1];
    for (int p = 0; p < P; ++p) {
        double sn, cs;
        sincos(logov[w * P + p].y, &sn, &cs);
        const double2 S = cmk(cs, sn);
        num = cadd(num, cmul(S, epair[w * P + p]));
        den = cadd(den, S);
    }
    acc[2 * w] = num;
    acc[2 * w + 1] = den;
}

// out[w] = E'_w, out[W + w] = R_w (zero for the walkers that do not count),
// out[2W] = sum_w W_w R_w E'_w, out[2W + 1] = sum_w W_w R_w; one block, fixed-order tree.
__global__ void __launch_bounds__(1024) meas_finish_kernel(int W, int rounds, const double* __restrict__ weight,
                                                           const double2* __restrict__ sumS0,
                                                           const int* __restrict__ alive,
                                                           const double2* __restrict__ acc, double2* out) {
    __shared__ double2 ra[1024], rb[1024];
    double2 A = cmk(0.0, 0.0), B = cmk(0.0, 0.0);
    for (int w = threadIdx.x; w < W; w += 1024) {
        double2 e = cmk(0.0, 0.0), R = cmk(0.0, 0.0);
        if (alive[w]) {
            const double2 den = acc[2 * w + 1];
            e = cdiv(acc[2 * w], den);
            R = cdiv(den, cmk(rounds * sumS0[w].x, rounds * sumS0[w].y));
            const double2 wr = cmk(weight[w] * R.x, weight[w] * R.y);
            A = cadd(A, cmul(wr, e));
            B = cadd(B, wr);
        }
        out[w] = e;
        out[W + w] = R;
    }
    ra[threadIdx.x] = A;
    rb[threadIdx.x] = B;
    __syncthreads();
    for (int off = 512; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            ra[threadIdx.x] = cadd(ra[threadIdx.x], ra[threadIdx.x + off]);
            rb[threadIdx.x] = cadd(rb[threadIdx.x], rb[threadIdx.x + off]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * W] = ra[0];
        out[2 * W + 1] = rb[0];
    }
}

cudaError_t meas_alive(cudaStream_t s, const Dims& d, double thr, const double* weight, const double2* sumS,
                       int* alive) {
    meas_alive_kernel<<<(d.W + 255) / 256, 256, 0, s>>>(d.W, thr, weight, sumS, alive);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t meas_accumulate(cudaStream_t s, const Dims& d, const double2* logov, const double2* epair,
                            const int* alive, double2* acc) {
    meas_accumulate_kernel<<<(d.W + 127) / 128, 128, 0, s>>>(d.W, d.P, logov, epair, alive, acc);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t meas_finish(cudaStream_t s, const Dims& d, int rounds, const double* weight, const double2* sumS0,
                        const int* alive, const double2* acc, double2* out) {
    meas_finish_kernel<<<1, 1024, 0, s>>>(d.W, rounds, weight, sumS0, alive, acc, out);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- step bookkeeping
// counters: [0] steps taken, [1] accepted total, [2] proposed total,
// [3] accepted this step, [4] proposed this step.
__global__ void step_end_kernel(int cap, const double* measured3, double* history, unsigned long long* counters) {
    unsigned long long st = counters[0];
    double* rec = history + 4 * (st % (unsigned long long)cap);
    rec[0] = measured3[0];
    rec[1] = measured3[1];
    rec[2] = measured3[2];
    rec[3] = (double)counters[3];
    counters[1] += counters[3];
    counters[2] += counters[4];
    counters[3] = 0;
    counters[4] = 0;
    counters[0] = st + 1;
}

cudaError_t step_end(cudaStream_t s, const StepParams& p, const double* measured3, double* history,
                     unsigned long long* counters) {
    step_end_kernel<<<1, 1, 0, s>>>(p.history_capacity, measured3, history, counters); count_launches(1);
    return cudaGetLastError();
}

__global__ void set_value_kernel(double* out, long long n, double v) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = v;
}
__global__ void set_int_kernel(int* out, long long n, int v) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = v;
}
cudaError_t set_value(cudaStream_t s, double* out, long long n, double v) {
    if (n > 0) { set_value_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, v); count_launches(1); }
    return cudaGetLastError();
}
cudaError_t set_int(cudaStream_t s, int* out, long long n, int v) {
    if (n > 0) { set_int_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, v); count_launches(1); }
    return cudaGetLastError();
}

}  // namespace afq
