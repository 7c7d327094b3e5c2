// Tensor-core (tcgen05) version of the fused contraction for the force bias and
// local energy, in split 16-bit arithmetic with FP32 accumulation.
//
// Same quantities as the FP64 kernel (Eq. (15), (16), (27) with Wick's theorem):
//   R_g = Phi^T X_g (X_0 = h, X_{g+1} = L_g), M_g,s = R_g[:n_s] Theta_s,
//   v_g = sum_s Tr M_g,s,  E_L = sum_s Tr M_0,s + 1/2 sum_g>0 [v_g^2 - sum_s Tr M_g,s^2].
// Two splits of every operand x into 16-bit parts x = hi + lo:
//  * BF16: hi = bf16(x), lo = bf16(x - hi); products hi*hi + hi*lo + lo*hi in one
//    FP32 accumulator (about 16 significant bits per operand).
//  * FP16 fixed point: every row of A and column of B is first scaled by a power
//    of two that puts its largest entry in [128, 256); then hi = rint(x) is an
//    integer with |hi| <= 256 (exact in FP16) and lo = fp16(x - hi), |lo| <= 1/2
//    (about 20 significant bits relative to the row's largest entry).  The
//    tensor cores truncate their FP32 accumulator toward zero after every MMA,
//    a bias that adds up over long sums; so hi*hi goes to its own accumulator,
//    where every partial sum is an integer below 2^23 (K <= 128) and therefore
//    exact, and hi*lo + lo*hi + lo*lo to a second one, about 2^-8 as large, whose
//    truncation error is below 2^-28 of the result.  The two are added with
//    round-to-nearest on the CUDA cores, and the exact scales are removed there.
//
// Mapping onto 128-row UMMA tiles (cta_group::1, kind::f16, both operands K-major,
// 128-byte swizzle):
//   GEMM1  D1[(g, j), (p, a)] = sum_i X_g[j, i] Phi_p[i, a]
//          A = GPT matrices X_g stacked (GPT = 128 / NPAD), streamed from a
//          pre-swizzled global image; B = Phi^T of the block's TP pairs (resident).
//   GEMM2  D2[(g, a), c]      = sum_j R_g,p[a, j] ThetaT_p[c, j]
//          A = R of GT consecutive g stacked (GT * n_up <= 128 rows), written by the
//          epilogue of GEMM1; B = Theta_p as [Re up | Im up | Re down | Im down]
//          (resident for the block's pairs).
// Accumulators live in tensor memory; traces are formed from D2 in FP32 and
// summed over a and g in FP64.  One block of 128 threads per TP pairs; thread 0
// issues the MMAs, all four warps run the epilogues on their tensor-memory lanes.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace afq {

constexpr int TC_THREADS = 128;
constexpr int TC_MAXTP = 32;

template <bool F16>
struct Half16;
template <>
struct Half16<false> {
    typedef __nv_bfloat16 T;
    static __device__ __forceinline__ T from(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ float to(T x) { return __bfloat162float(x); }
};
template <>
struct Half16<true> {
    typedef __half T;
    static __device__ __forceinline__ T from(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ float to(T x) { return __half2float(x); }
};

template <bool F16>
__device__ __forceinline__ void split16(float x, uint8_t* hi_base, uint8_t* lo_base, uint32_t off) {
    typedef Half16<F16> H;
    typename H::T hi, lo;
    if (F16) {
        float h = rintf(x);
        hi = H::from(h);
        lo = H::from(x - h);
    } else {
        hi = H::from(x);
        lo = H::from(x - H::to(hi));
    }
    *reinterpret_cast<typename H::T*>(hi_base + off) = hi;
    *reinterpret_cast<typename H::T*>(lo_base + off) = lo;
}
template <bool F16>
__device__ __forceinline__ void split16d(double x, uint8_t* hi_base, uint8_t* lo_base, uint32_t off) {
    typedef Half16<F16> H;
    typename H::T hi, lo;
    if (F16) {
        double h = rint(x);
        hi = H::from((float)h);
        lo = H::from((float)(x - h));
    } else {
        hi = H::from((float)x);
        lo = H::from((float)(x - (double)H::to(hi)));
    }
    *reinterpret_cast<typename H::T*>(hi_base + off) = hi;
    *reinterpret_cast<typename H::T*>(lo_base + off) = lo;
}
// Exponent e with max * 2^e in [128, 256) (0 for max = 0 or in BF16 mode).
template <bool F16>
__device__ __forceinline__ int scale_exp(float m) {
    if (!F16 || !(m > 0.f) || !isfinite(m)) return 0;
    return 7 - ilogbf(m);
}

// Power-of-two exponent of each matrix X_0 = h, X_1.. = L_g (FP16 mode only):
// one block per matrix.
template <bool F16>
__global__ void lt_scale_kernel(int N, int G1, const double* __restrict__ h, const double* __restrict__ L, int* lexp) {
    __shared__ float red[256];
    int g = blockIdx.x;
    float m = 0.f;
    if (g < G1) {
        const double* X = g == 0 ? h : L + (long long)(g - 1) * N * N;
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) m = fmaxf(m, (float)fabs(X[e]));
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + off]);
        __syncthreads();
    }
    if (threadIdx.x == 0) lexp[g] = scale_exp<F16>(red[0]);
}

// Image of X_0 = h, X_1.. = L_g (each times 2^lexp[g]) in the shared-memory
// layout of the A operand of GEMM1: tile t holds X_{t*GPT} .. X_{t*GPT + GPT - 1}
// as 128 rows (g, j); each of its NKB K blocks of 64 columns is 16 KB of hi
// followed by 16 KB of lo.  Matrices past the last X are zero.
template <bool F16>
__global__ void prepare_lt_kernel(int N, int NPAD, int G1, int n_tiles, const double* __restrict__ h,
                                  const double* __restrict__ L, const int* __restrict__ lexp, uint8_t* __restrict__ out) {
    int GPT = 128 / NPAD, NKB = NPAD / 64;
    long long total = (long long)n_tiles * NKB * 128 * 64;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        long long tk = e / (128 * 64);
        int rem = (int)(e - tk * 128 * 64);
        int row = rem / 64, kk = rem % 64;
        int t = (int)(tk / NKB), kb = (int)(tk % NKB);
        int g = t * GPT + row / NPAD, j = row % NPAD, i = kb * 64 + kk;
        double x = 0.0;
        if (g < G1 && j < N && i < N) {
            x = (g == 0) ? h[(long long)j * N + i] : L[((long long)(g - 1) * N + j) * N + i];
            x = ldexp(x, lexp[g]);
        }
        uint8_t* img = out + tk * 32768;
        split16d<F16>(x, img, img + 16384, tc::sw128_offset(128, row, kk));
    }
}

struct TcShape {
    int NPAD, GPT, NKB, TP, GT, NB1, NB2, c1col, d2col;
    size_t smem;
};

constexpr int TC_MAXSCALE_B2 = 512;   // TP * NB2 column scales of the Theta tiles

template <int NPAD, bool F16>
__global__ void __launch_bounds__(TC_THREADS, 1)
    contract_tc_kernel(int N, int nu, int nd, int G, int TP, int GT, int NB1, int NB2, int c1col, int d2col, long long pairs,
                       const uint4* __restrict__ Lt, const int* __restrict__ lexp, const double* __restrict__ Phi,
                       const double2* __restrict__ Theta, double2* __restrict__ vpair, double2* __restrict__ epair,
                       int* status) {
    constexpr int GPT = 128 / NPAD;
    constexpr int NKB = NPAD / 64;
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const size_t b1_bytes = (size_t)NB1 * NPAD * 2, b2_bytes = (size_t)NB2 * NPAD * 2;
    uint8_t* B1h = sm;
    uint8_t* B1l = B1h + b1_bytes;
    uint8_t* B2 = B1l + b1_bytes;                         // pair p: hi at 2p*b2, lo at (2p+1)*b2
    uint8_t* A1h = B2 + 2 * (size_t)TP * b2_bytes;
    uint8_t* A1l = A1h + 16384;
    uint8_t* A2h = A1l + 16384;
    uint8_t* A2l = A2h + (size_t)128 * NPAD * 2;
    float* Ms = reinterpret_cast<float*>(A1h);             // epilogue-2 staging over A1 and A2
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ float2 red_tr[TC_THREADS], red_ex[TC_THREADS];
    __shared__ double2 red_c[TC_THREADS];
    __shared__ double2 eacc[TC_MAXTP];
    __shared__ int sPhi[256];                 // column exponents of B1 (rows (p, a))
    __shared__ int sTh[TC_MAXSCALE_B2];       // column exponents of B2, per pair
    __shared__ unsigned rowmax[128];          // |R| maxima of the A2 rows (float bits)
    __shared__ int sR[128];                   // row exponents of A2

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = nu + nd;
    const long long pair0 = (long long)blockIdx.x * TP;
    const int np = (int)min((long long)TP, pairs - pair0);
    const int G1 = G + 1;
    const int S = nu * nu + nd * nd;

    if (warp == 0) {
        tc::tmem_alloc(&tslot, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_fence_init();
    }
    if (tid < TC_MAXTP) eacc[tid] = cmk(0.0, 0.0);
    // column exponents of B1 = Phi^T (row (p, a) of the operand) and of B2 = Theta^T
    for (int r = tid; r < NB1; r += TC_THREADS) {
        int p = r / nu, a = r % nu;
        float m = 0.f;
        if (F16 && p < np)
            for (int i = 0; i < N; ++i) m = fmaxf(m, (float)fabs(Phi[(pair0 + p) * (long long)N * nu + (long long)i * nu + a]));
        sPhi[r] = scale_exp<F16>(m);
    }
    for (int q = tid; q < TP * NB2; q += TC_THREADS) {
        int p = q / NB2, c = q % NB2;
        float m = 0.f;
        if (F16 && p < np && c < 2 * nt) {
            int col, im;
            if (c < 2 * nu) { col = c % nu; im = c >= nu; }
            else { int qq = c - 2 * nu; col = nu + qq % nd; im = qq >= nd; }
            const double2* Th = Theta + (pair0 + p) * (long long)N * nt;
            for (int j = 0; j < N; ++j) {
                double2 t = Th[(long long)j * nt + col];
                m = fmaxf(m, (float)fabs(im ? t.y : t.x));
            }
        }
        sTh[q] = scale_exp<F16>(m);
    }
    __syncthreads();
    // B1: Phi^T of the block's pairs, rows (p, a), K = i
    for (int e = tid; e < NB1 * NPAD; e += TC_THREADS) {
        int r = e / NPAD, i = e % NPAD;
        int p = r / nu, a = r % nu;
        double x = 0.0;
        if (p < np && i < N) x = ldexp(Phi[(pair0 + p) * (long long)N * nu + (long long)i * nu + a], sPhi[r]);
        split16d<F16>(x, B1h, B1l, tc::sw128_offset(NB1, r, i));
    }
    // B2: Theta_p^T as rows c = [Re up | Im up | Re down | Im down], K = j
    for (int p = 0; p < TP; ++p) {
        uint8_t* bh = B2 + 2 * (size_t)p * b2_bytes;
        uint8_t* bl = bh + b2_bytes;
        const double2* Th = Theta + (pair0 + p) * (long long)N * nt;
        for (int e = tid; e < NB2 * NPAD; e += TC_THREADS) {
            int c = e / NPAD, j = e % NPAD;
            double x = 0.0;
            if (p < np && j < N && c < 2 * nt) {
                int col, im;
                if (c < 2 * nu) { col = c % nu; im = c >= nu; }
                else { int q = c - 2 * nu; col = nu + q % nd; im = q >= nd; }
                double2 t = Th[(long long)j * nt + col];
                x = ldexp(im ? t.y : t.x, sTh[p * NB2 + c]);
            }
            split16d<F16>(x, bh, bl, tc::sw128_offset(NB2, c, j));
        }
    }
    // A2 starts zero (rows past GT * nu only ever feed D2 rows that are not read)
    for (int e = tid; e < 128 * NPAD * 2 * 2 / 16; e += TC_THREADS) reinterpret_cast<uint4*>(A2h)[e] = make_uint4(0, 0, 0, 0);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const uint32_t id1 = F16 ? tc::idesc_f16_f32(128, NB1) : tc::idesc_bf16_f32(128, NB1);
    const uint32_t id2 = F16 ? tc::idesc_f16_f32(128, NB2) : tc::idesc_bf16_f32(128, NB2);
    uint32_t phase = 0;
    bool failed = false;
    const int tiles_per_block = GT / GPT;
    const int n_blocks = (G1 + GT - 1) / GT;
    const int gs = tid / NPAD, jrow = tid % NPAD;       // this thread's D1 lane: (matrix in tile, row j)

    for (int gb = 0; gb < n_blocks && !failed; ++gb) {
        // ---- GEMM1 for the GT matrices of this block
        for (int k = 0; k < tiles_per_block && !failed; ++k) {
            const long long t = (long long)gb * tiles_per_block + k;
            for (int kb = 0; kb < NKB; ++kb) {
                const uint4* src = Lt + (t * NKB + kb) * 2048;
                for (int q = tid; q < 2048; q += TC_THREADS) reinterpret_cast<uint4*>(A1h)[q] = src[q];
                tc::fence_proxy_async();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
                if (tid == 0) {
                    const uint32_t d = taddr + (uint32_t)(k * NB1);
                    const uint32_t dc = taddr + (uint32_t)c1col;     // correction accumulator (FP16 mode)
#pragma unroll
                    for (int ss = 0; ss < 4; ++ss) {
                        uint64_t ah = tc::desc_sw128(tc::smem_u32(A1h) + ss * 32);
                        uint64_t al = tc::desc_sw128(tc::smem_u32(A1l) + ss * 32);
                        uint64_t bh = tc::desc_sw128(tc::smem_u32(B1h) + kb * NB1 * 128 + ss * 32);
                        uint64_t bl = tc::desc_sw128(tc::smem_u32(B1l) + kb * NB1 * 128 + ss * 32);
                        const uint32_t first = (kb > 0 || ss > 0) ? 1u : 0u;
                        tc::mma_f16(d, ah, bh, id1, first);
                        if (F16) {
                            tc::mma_f16(dc, ah, bl, id1, first);
                            tc::mma_f16(dc, al, bh, id1, 1u);
                            tc::mma_f16(dc, al, bl, id1, 1u);
                        } else {
                            tc::mma_f16(d, ah, bl, id1, 1u);
                            tc::mma_f16(d, al, bh, id1, 1u);
                        }
                    }
                    tc::mma_commit(&bar);
                }
                __syncwarp();
                bool ok = tc::mbar_wait(&bar, phase);
                phase ^= 1;
                if (__syncthreads_or(!ok)) { failed = true; break; }
                tc::fence_after_sync();
            }
            if (F16 && !failed) {
                // D1 tile += correction accumulator (round to nearest), so the
                // correction columns can take the next tile
                for (int c0 = 0; c0 < NB1; c0 += 16) {
                    float v[16], w[16];
                    tc::tmem_ld16(taddr + lane_base + (uint32_t)(k * NB1 + c0), v);
                    tc::tmem_ld16(taddr + lane_base + (uint32_t)(c1col + c0), w);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] += w[q];
                    tc::tmem_st16(taddr + lane_base + (uint32_t)(k * NB1 + c0), v);
                }
                tc::tmem_st_wait();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
            }
        }
        if (failed) break;
        // ---- per pair: epilogue 1 (R -> A2), GEMM2, epilogue 2 (traces)
        for (int p = 0; p < np && !failed; ++p) {
            // R_g,p[a, j] = D1[(g, j), (p, a)] * 2^-(lexp[g] + sPhi[p nu + a])
            if (F16) {
                if (tid < 128) rowmax[tid] = 0u;
                __syncthreads();
                for (int k = 0; k < tiles_per_block; ++k) {
                    const int gl = k * GPT + gs;
                    const int ge = gb * GT + gl;
                    const int le = ge < G1 ? lexp[ge] : 0;
                    for (int a0 = 0; a0 < nu; a0 += 16) {
                        float v[16];
                        tc::tmem_ld16(taddr + lane_base + (uint32_t)(k * NB1 + p * nu + a0), v);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            int a = a0 + q;
                            if (a < nu) {   // uniform across the warp
                                float r = ldexpf(v[q], -(le + sPhi[p * nu + a]));
                                unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(r)));
                                if (lane == 0) atomicMax(&rowmax[gl * nu + a], m);
                            }
                        }
                    }
                }
                __syncthreads();
                if (tid < 128) sR[tid] = scale_exp<F16>(__uint_as_float(rowmax[tid]));
                __syncthreads();
            }
            for (int k = 0; k < tiles_per_block; ++k) {
                const int gl = k * GPT + gs;
                const int ge = gb * GT + gl;
                const int le = (F16 && ge < G1) ? lexp[ge] : 0;
                for (int a0 = 0; a0 < nu; a0 += 16) {
                    float v[16];
                    tc::tmem_ld16(taddr + lane_base + (uint32_t)(k * NB1 + p * nu + a0), v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        int a = a0 + q;
                        if (a < nu) {
                            float r = v[q];
                            if (F16) r = ldexpf(r, sR[gl * nu + a] - le - sPhi[p * nu + a]);
                            split16<F16>(r, A2h, A2l, tc::sw128_offset(128, gl * nu + a, jrow));
                        }
                    }
                }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (tid == 0) {
                const uint8_t* bh_base = B2 + 2 * (size_t)p * b2_bytes;
                const uint8_t* bl_base = bh_base + b2_bytes;
                const uint32_t d = taddr + (uint32_t)d2col;
                for (int s = 0; s < NPAD / 16; ++s) {
                    const uint32_t ka = (uint32_t)((s >> 2) * 128 * 128 + (s & 3) * 32);
                    const uint32_t kbo = (uint32_t)((s >> 2) * NB2 * 128 + (s & 3) * 32);
                    uint64_t ah = tc::desc_sw128(tc::smem_u32(A2h) + ka);
                    uint64_t al = tc::desc_sw128(tc::smem_u32(A2l) + ka);
                    uint64_t bh = tc::desc_sw128(tc::smem_u32(bh_base) + kbo);
                    uint64_t bl = tc::desc_sw128(tc::smem_u32(bl_base) + kbo);
                    const uint32_t first = s > 0 ? 1u : 0u;
                    tc::mma_f16(d, ah, bh, id2, first);
                    if (F16) {
                        const uint32_t dc = d + (uint32_t)NB2;
                        tc::mma_f16(dc, ah, bl, id2, first);
                        tc::mma_f16(dc, al, bh, id2, 1u);
                        tc::mma_f16(dc, al, bl, id2, 1u);
                    } else {
                        tc::mma_f16(d, ah, bl, id2, 1u);
                        tc::mma_f16(d, al, bh, id2, 1u);
                    }
                }
                tc::mma_commit(&bar);
            }
            __syncwarp();
            bool ok = tc::mbar_wait(&bar, phase);
            phase ^= 1;
            if (__syncthreads_or(!ok)) { failed = true; break; }
            tc::fence_after_sync();
            // epilogue 2: M rows to shared memory (A1/A2 are free until the next GEMM)
            const int r = tid;
            const int gbl = r / nu, a = r % nu;
            const bool row_ok = r < GT * nu;
            const int er = (F16 && row_ok) ? sR[r] : 0;
            for (int c0 = 0; c0 < NB2; c0 += 16) {
                float v[16];
                tc::tmem_ld16(taddr + lane_base + (uint32_t)(d2col + c0), v);
                if (F16) {
                    float w[16];
                    tc::tmem_ld16(taddr + lane_base + (uint32_t)(d2col + NB2 + c0), w);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] += w[q];
                } else {
                    tc::tmem_ld_wait();
                }
                if (row_ok) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        int c = c0 + q;
                        float x = v[q];
                        if (F16 && c < 2 * nt) x = ldexpf(x, -(er + sTh[p * NB2 + c]));
                        if (c < 2 * nu) {
                            int b = c % nu, im = c >= nu;
                            Ms[2 * (gbl * S + a * nu + b) + im] = x;
                        } else if (c < 2 * nt && a < nd) {
                            int qq = c - 2 * nu;
                            int b = qq % nd, im = qq >= nd;
                            Ms[2 * (gbl * S + nu * nu + a * nd + b) + im] = x;
                        }
                    }
                }
            }
            tc::fence_before_sync();
            __syncthreads();
            if (row_ok) {
                const float* Mu = Ms + 2 * (gbl * S);
                const float* Md = Mu + 2 * nu * nu;
                float trx = Mu[2 * (a * nu + a)], try_ = Mu[2 * (a * nu + a) + 1];
                float exx = 0.f, exy = 0.f;
                for (int b = 0; b < nu; ++b) {
                    float x1 = Mu[2 * (a * nu + b)], y1 = Mu[2 * (a * nu + b) + 1];
                    float x2 = Mu[2 * (b * nu + a)], y2 = Mu[2 * (b * nu + a) + 1];
                    exx = fmaf(x1, x2, fmaf(-y1, y2, exx));
                    exy = fmaf(x1, y2, fmaf(y1, x2, exy));
                }
                if (a < nd) {
                    trx += Md[2 * (a * nd + a)];
                    try_ += Md[2 * (a * nd + a) + 1];
                    for (int b = 0; b < nd; ++b) {
                        float x1 = Md[2 * (a * nd + b)], y1 = Md[2 * (a * nd + b) + 1];
                        float x2 = Md[2 * (b * nd + a)], y2 = Md[2 * (b * nd + a) + 1];
                        exx = fmaf(x1, x2, fmaf(-y1, y2, exx));
                        exy = fmaf(x1, y2, fmaf(y1, x2, exy));
                    }
                }
                red_tr[r] = make_float2(trx, try_);
                red_ex[r] = make_float2(exx, exy);
            }
            __syncthreads();
            if (tid < GT) {
                double2 tr = cmk(0.0, 0.0), ex = cmk(0.0, 0.0);
                for (int aa = 0; aa < nu; ++aa) {
                    float2 x = red_tr[tid * nu + aa], y = red_ex[tid * nu + aa];
                    tr.x += x.x; tr.y += x.y;
                    ex.x += y.x; ex.y += y.y;
                }
                const int ge = gb * GT + tid;    // index into (h, L_0, L_1, ...)
                double2 c = cmk(0.0, 0.0);
                if (ge == 0) {
                    c = tr;
                } else if (ge <= G) {
                    vpair[(pair0 + p) * (long long)G + (ge - 1)] = tr;
                    double2 t2 = cmul(tr, tr);
                    c = cmk(0.5 * (t2.x - ex.x), 0.5 * (t2.y - ex.y));
                }
                red_c[tid] = c;
            }
            __syncthreads();
            if (tid == 0) {
                double2 s = eacc[p];
                for (int q = 0; q < GT; ++q) s = cadd(s, red_c[q]);
                eacc[p] = s;
            }
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
        }
    }
    if (failed) {
        if (tid == 0) atomicOr(status, STATUS_TIMEOUT);
    } else if (tid < np) {
        epair[pair0 + tid] = eacc[tid];
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

// Tile shape for (N, n_up, n_dn): the deepest stack of Cholesky matrices in
// GEMM2 (GT * n_up <= 128 rows) and then the most pairs per block (TP) that fit
// tensor memory and shared memory.  Tensor-memory columns, in order: GT/GPT D1
// tiles of NB1, (FP16 mode) one correction tile of NB1, D2 of NB2, (FP16 mode)
// its correction of NB2.
static bool tc_shape(int N, int nu, int nd, bool f16, TcShape& s) {
    s.NPAD = N <= 64 ? 64 : (N <= 128 ? 128 : 0);
    if (!s.NPAD || nu < 1 || nu > 32 || nd > nu) return false;
    s.GPT = 128 / s.NPAD;
    s.NKB = s.NPAD / 64;
    s.NB2 = ((2 * (nu + nd) + 15) / 16) * 16;
    for (int gt = (128 / nu) / s.GPT * s.GPT; gt >= s.GPT; gt -= s.GPT) {
        const int tiles = gt / s.GPT;
        const size_t ms = (size_t)gt * (nu * nu + nd * nd) * 8;
        if (ms > 32768 + 2 * (size_t)128 * s.NPAD * 2) continue;
        for (int tp = TC_MAXTP; tp >= 1; --tp) {
            int nb1 = ((tp * nu + 15) / 16) * 16;
            if (nb1 > 256) continue;
            int c1 = tiles * nb1;
            int d2 = f16 ? c1 + nb1 : c1;
            int end = d2 + (f16 ? 2 * s.NB2 : s.NB2);
            if (end > 512 || d2 + 32 > 512) continue;   // the D1 reads of a pair run up to 31 columns past its start
            if (tp * s.NB2 > TC_MAXSCALE_B2) continue;
            size_t smem = 1024 + 2 * (size_t)nb1 * s.NPAD * 2 + 2 * (size_t)tp * s.NB2 * s.NPAD * 2 + 32768 +
                          2 * (size_t)128 * s.NPAD * 2;
            if (smem > 223000) continue;   // plus about 8.6 KB of static shared memory <= 227 KB
            s.GT = gt;
            s.TP = tp;
            s.NB1 = nb1;
            s.c1col = c1;
            s.d2col = d2;
            s.smem = smem < 120 * 1024 ? 120 * 1024 : smem;   // one block per SM (it holds all 512 columns)
            return true;
        }
    }
    return false;
}

bool contract_tc_supported(int N, int nu, int nd, bool f16) {
    TcShape s;
    return tc_shape(N, nu, nd, f16, s);
}

size_t contract_tc_image_bytes(int N, int nu, int nd, int G, bool f16) {
    TcShape s;
    if (!tc_shape(N, nu, nd, f16, s)) return 0;
    long long G1p = (long long)((G + 1 + s.GT - 1) / s.GT) * s.GT;
    long long tiles = G1p / s.GPT;
    return (size_t)tiles * s.NKB * 32768 + (size_t)G1p * sizeof(int);
}

// The split image of (h, L_g) and, after it, the per-matrix exponents.
cudaError_t contract_tc_prepare(cudaStream_t st, int N, int nu, int nd, int G, const double* h, const double* L,
                                void* image, bool f16) {
    TcShape s;
    if (!tc_shape(N, nu, nd, f16, s)) return cudaErrorInvalidValue;
    long long G1p = (long long)((G + 1 + s.GT - 1) / s.GT) * s.GT;
    int tiles = (int)(G1p / s.GPT);
    int* lexp = reinterpret_cast<int*>(static_cast<uint8_t*>(image) + (size_t)tiles * s.NKB * 32768);
    if (f16) {
        lt_scale_kernel<true><<<(unsigned)G1p, 256, 0, st>>>(N, G + 1, h, L, lexp); count_launches(1);
        prepare_lt_kernel<true><<<1024, 256, 0, st>>>(N, s.NPAD, G + 1, tiles, h, L, lexp, (uint8_t*)image); count_launches(1);
    } else {
        lt_scale_kernel<false><<<(unsigned)G1p, 256, 0, st>>>(N, G + 1, h, L, lexp); count_launches(1);
        prepare_lt_kernel<false><<<1024, 256, 0, st>>>(N, s.NPAD, G + 1, tiles, h, L, lexp, (uint8_t*)image); count_launches(1);
    }
    return cudaGetLastError();
}

template <int NPAD, bool F16>
static cudaError_t launch_tc(cudaStream_t st, const Dims& d, const TcShape& s, const void* image, const int* lexp,
                             const double* Phi, const double2* Theta, double2* vpair, double2* epair, int* status) {
    cudaError_t e = raise_smem_limit((const void*)contract_tc_kernel<NPAD, F16>, s.smem);
    if (e != cudaSuccess) return e;
    long long blocks = (d.pairs + s.TP - 1) / s.TP;
    contract_tc_kernel<NPAD, F16><<<(unsigned)blocks, TC_THREADS, s.smem, st>>>(
        d.N, d.nu, d.nd, d.G, s.TP, s.GT, s.NB1, s.NB2, s.c1col, s.d2col, d.pairs, (const uint4*)image, lexp, Phi, Theta, vpair,
        epair, status); count_launches(1);
    return cudaGetLastError();
}

cudaError_t contract_tc(cudaStream_t st, const Dims& d, const void* image, const double* Phi, const double2* Theta,
                        double2* vpair, double2* epair, int* status, bool f16) {
    TcShape s;
    if (!tc_shape(d.N, d.nu, d.nd, f16, s)) return cudaErrorInvalidValue;
    if (d.tc_tp > 0 && d.tc_tp < s.TP) {   // fewer pairs per block: same tensor-memory layout rules, less shared memory
        s.TP = d.tc_tp;
        s.NB1 = ((s.TP * d.nu + 15) / 16) * 16;
        s.c1col = (s.GT / s.GPT) * s.NB1;
        s.d2col = f16 ? s.c1col + s.NB1 : s.c1col;
        size_t smem = 1024 + 2 * (size_t)s.NB1 * s.NPAD * 2 + 2 * (size_t)s.TP * s.NB2 * s.NPAD * 2 + 32768 +
                      2 * (size_t)128 * s.NPAD * 2;
        s.smem = smem < 120 * 1024 ? 120 * 1024 : smem;
    }
    long long G1p = (long long)((d.G + 1 + s.GT - 1) / s.GT) * s.GT;
    const int* lexp = reinterpret_cast<const int*>(static_cast<const uint8_t*>(image) +
                                                   (size_t)(G1p / s.GPT) * s.NKB * 32768);
    if (s.NPAD == 64)
        return f16 ? launch_tc<64, true>(st, d, s, image, lexp, Phi, Theta, vpair, epair, status)
                   : launch_tc<64, false>(st, d, s, image, lexp, Phi, Theta, vpair, epair, status);
    return f16 ? launch_tc<128, true>(st, d, s, image, lexp, Phi, Theta, vpair, epair, status)
               : launch_tc<128, false>(st, d, s, image, lexp, Phi, Theta, vpair, epair, status);
}

}  // namespace afq
