// Learned Metropolis proposal for the paths' hidden variables.
//
// The paper lets the paths be updated by any proposal whose Metropolis
// acceptance keeps the sampled trial exact (Sec. III A, after Eq. (23)).  This
// one is a diagonal Gaussian conditioned on walker features:
//   f_k     = Re sum_s Tr[(Phi0_s^T phi_s)^-1 Phi0_s^T U_k phi_s]
//             (the gradient of log|<Phi(x)|phi>| at x = 0),
//   out     = W3 tanh(W2 tanh(W1 f + b1) + b2) + b3        (hidden width 256),
//   mu      = f + out[:K],  logv = clip(out[K:], -6, 3),
// trained on the paths' states by minimising the Gaussian negative
// log-likelihood with Adam.  Weights and activations enter the GEMMs in BF16
// with FP32 accumulation (tcgen05 MMAs, accumulators in tensor memory); master weights, Adam
// moments, biases and the head stay FP32.  Parameters are one flat FP32 vector:
// W1 (H x K), b1 (H), W2 (H x H), b2 (H), W3 (2K x H), b3 (2K), row-major.
#include <cuda_bf16.h>

#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace afq {

constexpr int MLP_H = 256;
constexpr float LOGV_MIN = -6.f, LOGV_MAX = 3.f;

long long mlp_n_params(int K) { return (long long)MLP_H * K + MLP_H + MLP_H * MLP_H + MLP_H + 2LL * K * MLP_H + 2 * K; }

// ---------------------------------------------------------------- GEMM (BF16 in, FP32 out)
// C[M x N] = A[M x K] B[K x N] on the fifth-generation tensor cores: one block of
// 128 threads per 128 x 128 tile of C (tcgen05.mma.cta_group::1.kind::f16, BF16
// operands, FP32 accumulator in tensor memory).  For each K chunk of 64 the block
// copies the A tile (128 rows) and the B tile (up to 128 columns) into shared
// memory as K-major operands in the 128-byte swizzled layout, converting the
// stored layout on the way: A row-major (A[m][k] at A[m lda + k]) or
// column-major (at A[k lda + m]); B column-major (B[k][n] at B[n ldb + k], the
// transposed weights) or row-major (at B[k ldb + n]).  Thread 0 issues the
// chunk's MMAs and commits them to an mbarrier (bounded wait); the four warps then
// read their 32 rows of the accumulator.  M, N, K multiples of 16; rows and
// columns past M and N are zero in the operands and not stored.
template <bool A_RM, bool B_RM>
__global__ void __launch_bounds__(128) mlp_gemm_kernel(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                       int lda, const __nv_bfloat16* __restrict__ B, int ldb,
                                                       float* __restrict__ C, int ldc, int* status, uint32_t lim) {
    __shared__ __align__(1024) uint8_t sa[128 * 128];   // 128 rows x 64 K values (bf16)
    __shared__ __align__(1024) uint8_t sb[128 * 128];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * 128, n0 = blockIdx.x * 128;
    const int bn = min(128, N - n0);                      // columns of this tile, a multiple of 16
    if (warp == 0) {
        tc::tmem_alloc(&tslot, 128);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_fence_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    const uint32_t idesc = tc::idesc_bf16_f32(128, bn);
    bool failed = false;
    int phase = 0;
    for (int k0 = 0; k0 < K; k0 += 64) {
        const int kc = min(64, K - k0);
        // operand tiles: unit u = (row r, 8 consecutive k) as one 16-byte store
        for (int u = tid; u < 128 * 8; u += 128) {
            const int r = u >> 3, ku = (u & 7) * 8;
            uint16_t va[8], vb[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int k = k0 + ku + t, m = m0 + r, n = n0 + r;
                va[t] = 0;
                vb[t] = 0;
                if (ku + t < kc) {
                    if (m < M) va[t] = __bfloat16_as_ushort(A_RM ? A[(size_t)m * lda + k] : A[(size_t)k * lda + m]);
                    if (r < bn) vb[t] = __bfloat16_as_ushort(B_RM ? B[(size_t)k * ldb + n] : B[(size_t)n * ldb + k]);
                }
            }
            const uint32_t off = tc::sw128_offset(128, r, ku);
            *reinterpret_cast<uint4*>(sa + off) = make_uint4((uint32_t)va[0] | ((uint32_t)va[1] << 16),
                                                             (uint32_t)va[2] | ((uint32_t)va[3] << 16),
                                                             (uint32_t)va[4] | ((uint32_t)va[5] << 16),
                                                             (uint32_t)va[6] | ((uint32_t)va[7] << 16));
            *reinterpret_cast<uint4*>(sb + off) = make_uint4((uint32_t)vb[0] | ((uint32_t)vb[1] << 16),
                                                             (uint32_t)vb[2] | ((uint32_t)vb[3] << 16),
                                                             (uint32_t)vb[4] | ((uint32_t)vb[5] << 16),
                                                             (uint32_t)vb[6] | ((uint32_t)vb[7] << 16));
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t pa = tc::smem_u32(sa), pb = tc::smem_u32(sb);
            for (int s = 0; s < kc / 16; ++s)
                tc::mma_f16(taddr, tc::desc_sw128(pa + 32u * s), tc::desc_sw128(pb + 32u * s), idesc,
                            (k0 > 0 || s > 0) ? 1u : 0u);
            tc::mma_commit(&bar);
        }
        // the MMAs read the tiles: wait before the next chunk overwrites them
        const bool ok = tc::mbar_wait(&bar, (uint32_t)phase, lim);
        phase ^= 1;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        tc::fence_after_sync();
    }
    if (failed) {
        if (tid == 0) {
            atomicOr(status, STATUS_TIMEOUT);
            tc::mbar_wait(&bar, (uint32_t)(phase ^ 1), 1u << 22);   // the issued MMAs complete
        }
    } else {
        // warp w reads accumulator rows 32 w .. 32 w + 31 (its tensor-memory lane quadrant)
        const int m = m0 + 32 * warp + lane;
        for (int c0 = 0; c0 < bn; c0 += 16) {
            float v[16];
            tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            tc::tmem_ld_wait();
            if (m < M)
#pragma unroll
                for (int t = 0; t < 16; ++t) C[(size_t)m * ldc + n0 + c0 + t] = v[t];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 128);
}

template <bool A_RM, bool B_RM>
static void gemm16(cudaStream_t s, const Dims& d, const MlpBuffers& mb, int M, int N, int K, const __nv_bfloat16* A,
                   int lda, const __nv_bfloat16* B, int ldb, float* C, int ldc) {
    dim3 grid((unsigned)((N + 127) / 128), (unsigned)((M + 127) / 128));
    mlp_gemm_kernel<A_RM, B_RM><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, mb.status, d.wait_polls);
    count_launches(1);
}
// operand layouts of gemm16: row-major (RM) or column-major (CM), for A and for B
constexpr bool RM = true, CM = false;

// ---------------------------------------------------------------- elementwise kernels
// features f_w,k from Theta0 = phi (Phi0^T phi)^-1 and UPhi0[k] = U_k Phi0
__global__ void mlp_features_kernel(int N, int nu, int nd, int K, int Kp, const double2* __restrict__ Theta0,
                                    const double* __restrict__ UPhi0, float* featf, __nv_bfloat16* featb) {
    int w = blockIdx.x, nt = nu + nd;
    const double2* T = Theta0 + (size_t)w * N * nt;
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        double f = 0.0;
        if (k < K) {
            const double* UP = UPhi0 + (size_t)k * N * nu;
            for (int j = 0; j < N; ++j) {
                for (int a = 0; a < nu; ++a) f = fma(T[(size_t)j * nt + a].x, UP[(size_t)j * nu + a], f);
                for (int a = 0; a < nd; ++a) f = fma(T[(size_t)j * nt + nu + a].x, UP[(size_t)j * nu + a], f);
            }
        }
        featf[(size_t)w * Kp + k] = (float)f;
        featb[(size_t)w * Kp + k] = __float2bfloat16_rn((float)f);
    }
}

// H = tanh(Z + b) for rows < rows_live (others 0), FP32 and BF16 copies
__global__ void mlp_bias_tanh_kernel(int rows, int rows_live, int N, const float* __restrict__ Z, const float* __restrict__ b,
                                     float* Hf, __nv_bfloat16* Hb) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)rows * N) return;
    int r = (int)(e / N), c = (int)(e % N);
    float h = r < rows_live ? tanhf(Z[e] + b[c]) : 0.f;
    Hf[e] = h;
    Hb[e] = __float2bfloat16_rn(h);
}

// mu = f + out[:K] + b3[:K]; logv = clip(out[Kp:Kp+K] + b3[K:])
__global__ void mlp_head_kernel(int rows_live, int K, int Kp, const float* __restrict__ out, const float* __restrict__ b3,
                                const float* __restrict__ featf, float* mu, float* logv, float* logv_raw) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)rows_live * K) return;
    int w = (int)(e / K), k = (int)(e % K);
    float m = featf[(size_t)w * Kp + k] + out[(size_t)w * 2 * Kp + k] + b3[k];
    float lr = out[(size_t)w * 2 * Kp + Kp + k] + b3[K + k];
    mu[e] = m;
    logv_raw[e] = lr;
    logv[e] = fminf(fmaxf(lr, LOGV_MIN), LOGV_MAX);
}

// d loss / d out and the per-walker loss, loss = 1/(B P) sum 1/2 [(x - mu)^2 / v + logv]
__global__ void mlp_loss_grad_kernel(int B, int P, int K, int Kp, const double* __restrict__ x, const float* __restrict__ mu,
                                     const float* __restrict__ logv, const float* __restrict__ logv_raw, float* doutf,
                                     __nv_bfloat16* doutb, double* loss_part) {
    __shared__ double red[256];
    int w = blockIdx.x;
    double scale = 1.0 / ((double)B * P);
    double lsum = 0.0;
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        float dm = 0.f, dl = 0.f;
        if (k < K) {
            double m = mu[(size_t)w * K + k], lv = logv[(size_t)w * K + k], iv = exp(-lv);
            double gm = 0.0, gl = 0.0;
            for (int p = 0; p < P; ++p) {
                double r = x[((size_t)w * P + p) * K + k] - m;
                gm -= r * iv;
                gl += 0.5 * (1.0 - r * r * iv);
                lsum += 0.5 * (r * r * iv + lv);
            }
            float raw = logv_raw[(size_t)w * K + k];
            dm = (float)(gm * scale);
            dl = (raw > LOGV_MIN && raw < LOGV_MAX) ? (float)(gl * scale) : 0.f;
        }
        doutf[(size_t)w * 2 * Kp + k] = dm;
        doutf[(size_t)w * 2 * Kp + Kp + k] = dl;
        doutb[(size_t)w * 2 * Kp + k] = __float2bfloat16_rn(dm);
        doutb[(size_t)w * 2 * Kp + Kp + k] = __float2bfloat16_rn(dl);
    }
    red[threadIdx.x] = lsum;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[w] = red[0] * scale;
}

// dZ = dH (1 - H^2) for rows < rows_live (others 0)
__global__ void mlp_tanh_back_kernel(int rows, int rows_live, int N, const float* __restrict__ dH, const float* __restrict__ Hf,
                                     float* dZf, __nv_bfloat16* dZb) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)rows * N) return;
    int r = (int)(e / N);
    float h = Hf[e];
    float d = r < rows_live ? dH[e] * (1.f - h * h) : 0.f;
    dZf[e] = d;
    dZb[e] = __float2bfloat16_rn(d);
}

// out[c] = sum over rows < rows_live of M[r][c] (fixed order)
__global__ void mlp_colsum_kernel(int rows_live, int N, int ld, const float* __restrict__ Mx, float* out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    float s = 0.f;
    for (int r = 0; r < rows_live; ++r) s += Mx[(size_t)r * ld + c];
    out[c] = s;
}

// flat gradient (oracle layout) from the padded weight gradients and bias sums
__global__ void mlp_gather_grad_kernel(int K, int Kp, const float* __restrict__ gW1p, const float* __restrict__ gb1,
                                       const float* __restrict__ gW2, const float* __restrict__ gb2,
                                       const float* __restrict__ gW3p, const float* __restrict__ gb3p, float* grad) {
    const int H = MLP_H;
    long long n = (long long)H * K + H + H * H + H + 2LL * K * H + 2 * K;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        long long q = e;
        float v;
        if (q < (long long)H * K) { v = gW1p[(q / K) * Kp + q % K]; }
        else if ((q -= (long long)H * K) < H) { v = gb1[q]; }
        else if ((q -= H) < (long long)H * H) { v = gW2[q]; }
        else if ((q -= (long long)H * H) < H) { v = gb2[q]; }
        else if ((q -= H) < 2LL * K * H) {
            long long r = q / H, c = q % H;
            long long pr = r < K ? r : Kp + (r - K);
            v = gW3p[pr * H + c];
        } else {
            q -= 2LL * K * H;
            v = q < K ? gb3p[q] : gb3p[Kp + (q - K)];
        }
        grad[e] = v;
    }
}

// BF16 padded weight matrices from the flat FP32 parameters
__global__ void mlp_pack_kernel(int K, int Kp, const float* __restrict__ theta, __nv_bfloat16* W1b, __nv_bfloat16* W2b,
                                __nv_bfloat16* W3b) {
    const int H = MLP_H;
    long long n1 = (long long)H * Kp, n2 = (long long)H * H, n3 = 2LL * Kp * H;
    const float* W1 = theta;
    const float* W2 = W1 + (long long)H * K + H;
    const float* W3 = W2 + (long long)H * H + H;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n1 + n2 + n3; e += (long long)gridDim.x * blockDim.x) {
        if (e < n1) {
            long long h = e / Kp, k = e % Kp;
            W1b[e] = __float2bfloat16_rn(k < K ? W1[h * K + k] : 0.f);
        } else if (e < n1 + n2) {
            W2b[e - n1] = __float2bfloat16_rn(W2[e - n1]);
        } else {
            long long q = e - n1 - n2, r = q / H, c = q % H;
            float v = 0.f;
            if (r < K) v = W3[r * H + c];
            else if (r >= Kp && r < Kp + K) v = W3[(K + r - Kp) * H + c];
            W3b[q] = __float2bfloat16_rn(v);
        }
    }
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the flat parameters; the step
// count lives on the device so a captured step replays correctly.
__global__ void mlp_adam_kernel(long long n, float lr, float* theta, float* m, float* v, const float* __restrict__ g,
                                const unsigned long long* t_ctr) {
    double t = (double)(t_ctr[0] + 1);
    float c1 = (float)(1.0 - pow(0.9, t)), c2 = (float)(1.0 - pow(0.999, t));
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float gi = g[e];
        float mi = 0.9f * m[e] + 0.1f * gi;
        float vi = 0.999f * v[e] + 0.001f * gi * gi;
        m[e] = mi;
        v[e] = vi;
        theta[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    }
}
__global__ void mlp_count_kernel(unsigned long long* t_ctr) { t_ctr[0] += 1; }

// Deterministic initial parameters: weights N(0, 1/fan_in) from Philox (tag
// MLP_INIT, entity = parameter block), the output layer scaled by 1e-2 so the
// untrained proposal is N(f, I); biases 0.
__global__ void mlp_init_kernel(int K, uint64_t seed, float* theta) {
    const int H = MLP_H;
    long long nW1 = (long long)H * K, nW2 = (long long)H * H, nW3 = 2LL * K * H;
    long long o1 = 0, ob1 = nW1, o2 = ob1 + H, ob2 = o2 + nW2, o3 = ob2 + H, ob3 = o3 + nW3, n = ob3 + 2 * K;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float scale;
        if (e < ob1) scale = rsqrtf((float)K);
        else if (e < o2) scale = 0.f;
        else if (e < ob2) scale = rsqrtf((float)H);
        else if (e < o3) scale = 0.f;
        else if (e < ob3) scale = 1e-2f * rsqrtf((float)H);
        else scale = 0.f;
        double z = scale != 0.f ? normal_at(seed, TAG_MLP_INIT, 0, (uint32_t)(e >> 12), 0, (uint32_t)(e & 4095)) : 0.0;
        theta[e] = (float)(scale * z);
        (void)o1;
    }
}

__global__ void mlp_sum_kernel(int n, const double* __restrict__ part, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        out[0] = s;
    }
}

static unsigned grid_for(long long n) { return (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

// ---------------------------------------------------------------- host orchestration
cudaError_t mlp_prepare(cudaStream_t s, const Dims& d, const MlpBuffers& m, const double* U, const double* Phi0,
                        uint64_t seed) {
    // U_k Phi0 for all k: (K N x N) (N x n_up)
    gemm_nn_f64(s, d.K * d.N, d.nu, d.N, 1.0, U, d.N, Phi0, d.nu, 0.0, m.UPhi0, d.nu);
    mlp_init_kernel<<<grid_for(mlp_n_params(d.K)), 256, 0, s>>>(d.K, seed, m.theta); count_launches(1);
    cudaError_t e;
    if ((e = cudaMemsetAsync(m.adam_m, 0, sizeof(float) * mlp_n_params(d.K), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(m.adam_v, 0, sizeof(float) * mlp_n_params(d.K), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(m.counter, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(m.featf, 0, sizeof(float) * (size_t)m.Wp * m.Kp, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(m.featb, 0, sizeof(__nv_bfloat16) * (size_t)m.Wp * m.Kp, s)) != cudaSuccess) return e;
    return mlp_pack(s, d, m);
}

cudaError_t mlp_pack(cudaStream_t s, const Dims& d, const MlpBuffers& m) {
    long long n = (long long)MLP_H * m.Kp + MLP_H * MLP_H + 2LL * m.Kp * MLP_H;
    mlp_pack_kernel<<<grid_for(n), 256, 0, s>>>(d.K, m.Kp, m.theta, m.W1b, m.W2b, m.W3b); count_launches(1);
    return cudaGetLastError();
}

cudaError_t mlp_features(cudaStream_t s, const Dims& d, const MlpBuffers& m, const double* Phi0, const double2* phi,
                         int* status) {
    Dims t = d;
    for (int spin = 0; spin < 2; ++spin) {
        cudaError_t e = overlap_lu(s, t, spin, Phi0, 0, phi, m.logdet0, m.Theta0, nullptr, status, d.W, 1);
        if (e != cudaSuccess) return e;
    }
    mlp_features_kernel<<<d.W, 128, 0, s>>>(d.N, d.nu, d.nd, d.K, m.Kp, m.Theta0, m.UPhi0, m.featf, m.featb); count_launches(1);
    return cudaGetLastError();
}

// Forward for the first `rows` walkers (features already in featf / featb).
cudaError_t mlp_forward(cudaStream_t s, const Dims& d, const MlpBuffers& m, int rows) {
    const int H = MLP_H, Kp = m.Kp, R = (rows + 15) / 16 * 16;
    const float* b1 = m.theta + (long long)H * d.K;
    const float* b2 = b1 + H + (long long)H * H;
    const float* b3 = b2 + H + 2LL * d.K * H;
    gemm16<RM, CM>(s, d, m, R, H, Kp, m.featb, Kp, m.W1b, Kp, m.Zf, H);
    mlp_bias_tanh_kernel<<<grid_for((long long)R * H), 256, 0, s>>>(R, rows, H, m.Zf, b1, m.H1f, m.H1b); count_launches(1);
    gemm16<RM, CM>(s, d, m, R, H, H, m.H1b, H, m.W2b, H, m.Zf, H);
    mlp_bias_tanh_kernel<<<grid_for((long long)R * H), 256, 0, s>>>(R, rows, H, m.Zf, b2, m.H2f, m.H2b); count_launches(1);
    gemm16<RM, CM>(s, d, m, R, 2 * Kp, H, m.H2b, H, m.W3b, H, m.outf, 2 * Kp);
    mlp_head_kernel<<<grid_for((long long)rows * d.K), 256, 0, s>>>(rows, d.K, Kp, m.outf, b3, m.featf, m.mu, m.logv,
                                                                   m.logv_raw); count_launches(1);
    return cudaGetLastError();
}

// Loss and flat gradient for `rows` walkers with paths x (rows x P x K); with
// apply = true also one Adam step and the BF16 weights refreshed.
cudaError_t mlp_backward(cudaStream_t s, const Dims& d, const MlpBuffers& m, int rows, const double* x, float lr,
                         bool apply) {
    const int H = MLP_H, Kp = m.Kp, K = d.K, R = (rows + 15) / 16 * 16;
    mlp_loss_grad_kernel<<<rows, 256, 0, s>>>(rows, d.P, K, Kp, x, m.mu, m.logv, m.logv_raw, m.doutf, m.doutb,
                                              m.loss_part); count_launches(1);
    if (R > rows) {
        cudaError_t e = cudaMemsetAsync(m.doutf + (size_t)rows * 2 * Kp, 0, sizeof(float) * (size_t)(R - rows) * 2 * Kp, s);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(m.doutb + (size_t)rows * 2 * Kp, 0, sizeof(__nv_bfloat16) * (size_t)(R - rows) * 2 * Kp, s);
        if (e != cudaSuccess) return e;
    }
    mlp_sum_kernel<<<1, 32, 0, s>>>(rows, m.loss_part, m.loss); count_launches(1);
    // output layer: gW3 = dout^T H2, gb3 = colsum(dout), dH2 = dout W3
    gemm16<CM, RM>(s, d, m, 2 * Kp, H, R, m.doutb, 2 * Kp, m.H2b, H, m.gW3p, H);
    mlp_colsum_kernel<<<(2 * Kp + 255) / 256, 256, 0, s>>>(rows, 2 * Kp, 2 * Kp, m.doutf, m.gb3p); count_launches(1);
    gemm16<RM, RM>(s, d, m, R, H, 2 * Kp, m.doutb, 2 * Kp, m.W3b, H, m.dHf, H);
    mlp_tanh_back_kernel<<<grid_for((long long)R * H), 256, 0, s>>>(R, rows, H, m.dHf, m.H2f, m.dZf, m.dZb); count_launches(1);
    // second layer: gW2 = dZ2^T H1, gb2, dH1 = dZ2 W2
    gemm16<CM, RM>(s, d, m, H, H, R, m.dZb, H, m.H1b, H, m.gW2, H);
    mlp_colsum_kernel<<<1, 256, 0, s>>>(rows, H, H, m.dZf, m.gb2); count_launches(1);
    gemm16<RM, RM>(s, d, m, R, H, H, m.dZb, H, m.W2b, H, m.dHf, H);
    mlp_tanh_back_kernel<<<grid_for((long long)R * H), 256, 0, s>>>(R, rows, H, m.dHf, m.H1f, m.dZf, m.dZb); count_launches(1);
    // first layer: gW1 = dZ1^T f, gb1
    gemm16<CM, RM>(s, d, m, H, Kp, R, m.dZb, H, m.featb, Kp, m.gW1p, Kp);
    mlp_colsum_kernel<<<1, 256, 0, s>>>(rows, H, H, m.dZf, m.gb1); count_launches(1);
    long long n = mlp_n_params(K);
    mlp_gather_grad_kernel<<<grid_for(n), 256, 0, s>>>(K, Kp, m.gW1p, m.gb1, m.gW2, m.gb2, m.gW3p, m.gb3p, m.grad); count_launches(1);
    if (apply) {
        mlp_adam_kernel<<<grid_for(n), 256, 0, s>>>(n, lr, m.theta, m.adam_m, m.adam_v, m.grad, m.counter); count_launches(1);
        mlp_count_kernel<<<1, 1, 0, s>>>(m.counter); count_launches(1);
        return mlp_pack(s, d, m);
    }
    return cudaGetLastError();
}

}  // namespace afq

using namespace afq;

extern "C" int64_t afqmc_mlp_n_params(int K) { return K > 0 ? mlp_n_params(K) : 0; }

#define MK(call)                                                                                            \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return set_error(AFQMC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

static afqmc_status need_mlp(afqmc_ctx* ctx) {
    if (!ctx) return set_error(AFQMC_ERR_ARG, "ctx is NULL");
    if (ctx->cfg.proposal != AFQMC_PROPOSAL_MLP) return set_error(AFQMC_ERR_ARG, "the context has no learned proposal");
    return AFQMC_OK;
}

extern "C" afqmc_status afqmc_mlp_params(afqmc_ctx* ctx, float* params, int64_t n, int set) {
    afqmc_status st = need_mlp(ctx);
    if (st != AFQMC_OK) return st;
    if (!params || n != mlp_n_params(ctx->d.K)) return set_error(AFQMC_ERR_ARG, "need %lld parameters", mlp_n_params(ctx->d.K));
    MlpBuffers& m = ctx->ws.mlp;
    if (set) {
        MK(cudaMemcpyAsync(m.theta, params, sizeof(float) * n, cudaMemcpyHostToDevice, ctx->stream));
        MK(mlp_pack(ctx->stream, ctx->d, m));
    } else {
        MK(cudaMemcpyAsync(params, m.theta, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->stream));
    }
    MK(cudaStreamSynchronize(ctx->stream));
    return AFQMC_OK;
}

extern "C" afqmc_status afqmc_mlp_eval(afqmc_ctx* ctx, int B, const float* features, const double* x, float* mu_logv,
                                       double* loss, float* grad) {
    afqmc_status st = need_mlp(ctx);
    if (st != AFQMC_OK) return st;
    const Dims& d = ctx->d;
    if (B < 1 || B > d.W || !features || !x) return set_error(AFQMC_ERR_ARG, "need 1 <= B <= n_walkers and inputs");
    MlpBuffers& m = ctx->ws.mlp;
    cudaStream_t s = ctx->stream;
    const int R = (B + 15) / 16 * 16;
    std::vector<float> ff((size_t)R * m.Kp, 0.f);
    std::vector<__nv_bfloat16> fb((size_t)R * m.Kp, __float2bfloat16(0.f));
    for (int w = 0; w < B; ++w)
        for (int k = 0; k < d.K; ++k) {
            ff[(size_t)w * m.Kp + k] = features[(size_t)w * d.K + k];
            fb[(size_t)w * m.Kp + k] = __float2bfloat16(features[(size_t)w * d.K + k]);
        }
    MK(cudaMemcpyAsync(m.featf, ff.data(), ff.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    MK(cudaMemcpyAsync(m.featb, fb.data(), fb.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice, s));
    double* xs = ctx->ws.xprop;   // scratch of pairs * K doubles
    MK(cudaMemcpyAsync(xs, x, sizeof(double) * (size_t)B * d.P * d.K, cudaMemcpyHostToDevice, s));
    MK(mlp_forward(s, d, m, B));
    MK(mlp_backward(s, d, m, B, xs, 0.f, false));
    if (mu_logv) {
        std::vector<float> mu((size_t)B * d.K), lv((size_t)B * d.K);
        MK(cudaMemcpyAsync(mu.data(), m.mu, mu.size() * 4, cudaMemcpyDeviceToHost, s));
        MK(cudaMemcpyAsync(lv.data(), m.logv, lv.size() * 4, cudaMemcpyDeviceToHost, s));
        MK(cudaStreamSynchronize(s));
        for (int w = 0; w < B; ++w)
            for (int k = 0; k < d.K; ++k) {
                mu_logv[(size_t)w * 2 * d.K + k] = mu[(size_t)w * d.K + k];
                mu_logv[(size_t)w * 2 * d.K + d.K + k] = lv[(size_t)w * d.K + k];
            }
    }
    if (loss) MK(cudaMemcpyAsync(loss, m.loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (grad) MK(cudaMemcpyAsync(grad, m.grad, sizeof(float) * mlp_n_params(d.K), cudaMemcpyDeviceToHost, s));
    MK(cudaStreamSynchronize(s));
    ctx->measured = false;
    return AFQMC_OK;
}

extern "C" afqmc_status afqmc_mlp_state(afqmc_ctx* ctx, float* features, float* mu, float* logv) {
    afqmc_status st = need_mlp(ctx);
    if (st != AFQMC_OK) return st;
    const Dims& d = ctx->d;
    MlpBuffers& m = ctx->ws.mlp;
    cudaStream_t s = ctx->stream;
    if (features)
        MK(cudaMemcpy2DAsync(features, sizeof(float) * d.K, m.featf, sizeof(float) * m.Kp, sizeof(float) * d.K, d.W,
                             cudaMemcpyDeviceToHost, s));
    if (mu) MK(cudaMemcpyAsync(mu, m.mu, sizeof(float) * (size_t)d.W * d.K, cudaMemcpyDeviceToHost, s));
    if (logv) MK(cudaMemcpyAsync(logv, m.logv, sizeof(float) * (size_t)d.W * d.K, cudaMemcpyDeviceToHost, s));
    MK(cudaStreamSynchronize(s));
    return AFQMC_OK;
}
