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

constexpr int TC_THREADS = 256;
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
// x = hi + lo as the raw bits of two 16-bit values (same rules as split16).
template <bool F16>
__device__ __forceinline__ void split_bits(float x, uint16_t& hi, uint16_t& lo) {
    typedef Half16<F16> H;
    typename H::T h, l;
    if (F16) {
        const float r = rintf(x);
        h = H::from(r);
        l = H::from(x - r);
    } else {
        h = H::from(x);
        l = H::from(x - H::to(h));
    }
    hi = *reinterpret_cast<uint16_t*>(&h);
    lo = *reinterpret_cast<uint16_t*>(&l);
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
    int NPAD, GPT, NKB, TP, GT, T, NB1, NB2, S, c1col, d2col;
    size_t smem;
};

constexpr int TC_MAXSCALE_B2 = 512;   // TP * NB2 column scales of the Theta tiles
constexpr int TC_MAXSTAGES = 4;       // ring of streamed (h, L_g) operand units
constexpr uint32_t TC_UNIT = 32768;   // one unit: 128 rows x 64 K, hi then lo (16 KB each)
constexpr size_t TC_SMEM_MAX = 216 * 1024;   // dynamic shared memory (static use is about 10.1 KB of 227 KB)

// 2^e as a float, for |e| <= 126: exact scaling without ldexpf.
__device__ __forceinline__ float pow2f(int e) {
    e = max(-126, min(126, e));
    return __int_as_float((e + 127) << 23);
}
// Exponent that puts the largest entry of a row (its bits as an unsigned) in [128, 256).
__device__ __forceinline__ int row_exp(unsigned maxbits) {
    if (maxbits == 0u) return 0;
    int ex = (int)((maxbits >> 23) & 255u) - 127;
    return max(-100, min(100, 7 - ex));
}

// Per block: TP pairs, every g.  Warp roles: thread 0 issues the bulk copies of
// the (h, L_g) operand image into an S-stage ring and every MMA; all eight
// warps run the epilogues, warp w on tensor-memory lanes 32 (w % 4) .. +31.
//   GEMM1 of a block of GT matrices: T = GT / GPT tiles of 128 rows (g, j),
//     each accumulated in its own columns (F16 mode: hi*hi in one set, the
//     corrections in a second set), streamed unit by unit from the ring; a
//     stage is refilled as soon as the MMAs reading it have completed (so S
//     copies stay in flight), and the next block's first units load while the
//     per-pair epilogues run.
//   per pair: epilogue 1 (row maxima of R_g,p over j, then R scaled to
//     [128, 256) per row, split, stored as the A operand of GEMM2), GEMM2
//     against Theta_p, epilogue 2 (M to shared memory, traces, sums over a and g).
template <int NPAD, bool F16>
__global__ void __launch_bounds__(TC_THREADS, 1)
    contract_tc_kernel(int N, int nu, int nd, int G, int TP, int GT, int NB1, int NB2, int S, int c1col, int d2col,
                       long long pairs, const uint8_t* __restrict__ image, const int* __restrict__ lexp,
                       const double* __restrict__ Phi, const double2* __restrict__ Theta, double2* __restrict__ vpair,
                       double2* __restrict__ epair, int* status, uint32_t lim) {
    constexpr int GPT = 128 / NPAD;
    constexpr int NKB = NPAD / 64;
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint8_t* A1 = sm;                                          // S stages of one unit
    uint8_t* A2h = A1 + (size_t)S * TC_UNIT;
    uint8_t* A2l = A2h + (size_t)128 * NPAD * 2;
    float* Ms = reinterpret_cast<float*>(A2h);                // epilogue-2 staging, over A2
    uint8_t* B1h = A2l + (size_t)128 * NPAD * 2;
    const size_t b1_bytes = (size_t)NB1 * NPAD * 2, b2_bytes = (size_t)NB2 * NPAD * 2;
    uint8_t* B1l = B1h + b1_bytes;
    uint8_t* B2 = B1l + b1_bytes;                              // pair p: hi at 2p*b2, lo at (2p+1)*b2
    __shared__ uint64_t full_bar[TC_MAXSTAGES], empty_bar[TC_MAXSTAGES], done_bar, drain_bar;
    __shared__ uint32_t tslot;
    __shared__ int fail_flag;
    __shared__ unsigned rowmax[128];
    __shared__ float2 red_tr[2][128], red_ex[2][128];
    __shared__ float2 red_cf[128];
    __shared__ double2 eacc[TC_MAXTP];
    __shared__ int sPhi[256];                 // column exponents of B1 (rows (p, a))
    __shared__ int sTh[TC_MAXSCALE_B2];       // column exponents of B2, per pair

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int nt = nu + nd;
    const long long pair0 = (long long)blockIdx.x * TP;
    const int np = (int)min((long long)TP, pairs - pair0);
    const int G1 = G + 1;
    const int T = GT / GPT;
    const int n_gb = (G1 + GT - 1) / GT;
    const int total = n_gb * T * NKB;                          // units of the image, in order

    if (warp == 0) {
        tc::tmem_alloc(&tslot, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            tc::mbar_init(&full_bar[q], 1);
            tc::mbar_init(&empty_bar[q], 1);
        }
        tc::mbar_init(&done_bar, 1);
        tc::mbar_init(&drain_bar, 1);
        tc::mbar_fence_init();
        fail_flag = 0;
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
    // the first S units of the operand image start loading now
    int loaded = 0;   // units whose copies were issued (meaningful in thread 0)
    if (tid == 0) {
        for (; loaded < S && loaded < total; ++loaded) {
            tc::mbar_arrive_expect_tx(&full_bar[loaded], TC_UNIT);
            tc::bulk_g2s(A1 + (size_t)loaded * TC_UNIT, image + (size_t)loaded * TC_UNIT, TC_UNIT, &full_bar[loaded]);
        }
    }
    // B1: Phi^T of the block's pairs, rows (p, a), K = i
    for (int e = tid; e < NB1 * NPAD; e += TC_THREADS) {
        int r = e / NPAD, i = e % NPAD;
        int p = r / nu, a = r % nu;
        float x = 0.f;
        if (p < np && i < N) x = (float)Phi[(pair0 + p) * (long long)N * nu + (long long)i * nu + a] * pow2f(sPhi[r]);
        split16<F16>(x, B1h, B1l, tc::sw128_offset(NB1, r, i));
    }
    // B2: Theta_p^T as rows c = [Re up | Im up | Re down | Im down], K = j
    for (int p = 0; p < TP; ++p) {
        uint8_t* bh = B2 + 2 * (size_t)p * b2_bytes;
        uint8_t* bl = bh + b2_bytes;
        const double2* Th = Theta + (pair0 + p) * (long long)N * nt;
        for (int e = tid; e < NB2 * NPAD; e += TC_THREADS) {
            int c = e / NPAD, j = e % NPAD;
            float x = 0.f;
            if (p < np && j < N && c < 2 * nt) {
                int col, im;
                if (c < 2 * nu) { col = c % nu; im = c >= nu; }
                else { int q = c - 2 * nu; col = nu + q % nd; im = q >= nd; }
                double2 t = Th[(long long)j * nt + col];
                x = (float)(im ? t.y : t.x) * pow2f(sTh[p * NB2 + c]);
            }
            split16<F16>(x, bh, bl, tc::sw128_offset(NB2, c, j));
        }
    }
    // A2 starts zero (its rows past GT * nu only ever feed D2 rows that are not read)
    for (int e = tid; e < 128 * NPAD * 2 * 2 / 16; e += TC_THREADS) reinterpret_cast<uint4*>(A2h)[e] = make_uint4(0, 0, 0, 0);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
    const uint32_t id1 = F16 ? tc::idesc_f16_f32(128, NB1) : tc::idesc_bf16_f32(128, NB1);
    const uint32_t id2 = F16 ? tc::idesc_f16_f32(128, NB2) : tc::idesc_bf16_f32(128, NB2);
    uint32_t done_phase = 0;
    bool failed = false;
    int consumed = 0;                                         // units whose MMAs were issued
    const int Lrow = 32 * quarter + lane;                      // this thread's tensor-memory lane
    const int g_in_tile = Lrow / NPAD, jrow = Lrow % NPAD;     // D1 row (matrix in tile, j)

    // Issue the copy of the next unit into the stage freed by the MMAs of unit
    // loaded - S (thread 0 only; bounded wait).
    auto refill_upto = [&](int last_consumed) -> bool {
        while (loaded < total && loaded - S <= last_consumed) {
            const int v = loaded - S, st = loaded % S;
            if (v >= 0 && !tc::mbar_wait(&empty_bar[st], (uint32_t)((v / S) & 1), lim)) return false;
            tc::mbar_arrive_expect_tx(&full_bar[st], TC_UNIT);
            tc::bulk_g2s(A1 + (size_t)st * TC_UNIT, image + (size_t)loaded * TC_UNIT, TC_UNIT, &full_bar[st]);
            ++loaded;
        }
        return true;
    };

    for (int gb = 0; gb < n_gb && !failed; ++gb) {
        // ---- GEMM1 for the GT matrices of this block (thread 0 issues everything)
        if (tid == 0) {
            bool ok = true;
            for (int k = 0; k < T && ok; ++k) {
                for (int kb = 0; kb < NKB && ok; ++kb) {
                    const int u = consumed, st = u % S;
                    if (!tc::mbar_wait(&full_bar[st], (uint32_t)((u / S) & 1), lim)) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t sa = tc::smem_u32(A1 + (size_t)st * TC_UNIT);
                    const uint32_t d = taddr + (uint32_t)(k * NB1);
                    const uint32_t dc = taddr + (uint32_t)(c1col + k * NB1);
#pragma unroll
                    for (int ss = 0; ss < 4; ++ss) {
                        uint64_t ah = tc::desc_sw128(sa + ss * 32);
                        uint64_t al = tc::desc_sw128(sa + 16384 + ss * 32);
                        uint64_t bh = tc::desc_sw128(tc::smem_u32(B1h) + kb * NB1 * 128 + ss * 32);
                        uint64_t bl = tc::desc_sw128(tc::smem_u32(B1l) + kb * NB1 * 128 + ss * 32);
                        const uint32_t acc = (kb > 0 || ss > 0) ? 1u : 0u;
                        tc::mma_f16(d, ah, bh, id1, acc);
                        if (F16) {
                            tc::mma_f16(dc, ah, bl, id1, acc);
                            tc::mma_f16(dc, al, bh, id1, 1u);
                            tc::mma_f16(dc, al, bl, id1, 1u);
                        } else {
                            tc::mma_f16(d, ah, bl, id1, 1u);
                            tc::mma_f16(d, al, bh, id1, 1u);
                        }
                    }
                    tc::mma_commit(&empty_bar[st]);
                    ++consumed;
                    // refill this stage as soon as its MMAs (a fraction of a load's latency)
                    // are done, so S copies stay in flight
                    if (!refill_upto(u)) ok = false;
                }
            }
            if (ok) {
                tc::mma_commit(&done_bar);
                // prefetch the next block's first units while the pair epilogues run
                ok = refill_upto(consumed - 1);
            }
            if (!ok) fail_flag = 1;
        }
        __syncwarp();
        {
            bool ok = fail_flag == 0 && tc::mbar_wait(&done_bar, done_phase, lim);
            done_phase ^= 1;
            if (__syncthreads_or(!ok || fail_flag)) { failed = true; break; }
            tc::fence_after_sync();
        }
        // ---- per pair: epilogue 1 (R -> A2), GEMM2, epilogue 2 (traces)
        for (int p = 0; p < np && !failed; ++p) {
            // R_g,p[a, j] = D1[(g, j), (p, a)] * 2^-(lexp[g] + sPhi[p nu + a])
            if (F16) {
                if (tid < 128) rowmax[tid] = 0u;
                __syncthreads();
                for (int k = half; k < T; k += 2) {
                    const int gl = k * GPT + g_in_tile;
                    const int ge = gb * GT + gl;
                    const int le = ge < G1 ? lexp[ge] : 0;
                    for (int a0 = 0; a0 < nu; a0 += 16) {
                        float v[16], w[16];
                        tc::tmem_ld16(taddr + lane_base + (uint32_t)(k * NB1 + p * nu + a0), v);
                        tc::tmem_ld16(taddr + lane_base + (uint32_t)(c1col + k * NB1 + p * nu + a0), w);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int a = a0 + q;
                            if (a < nu) {   // uniform across the warp
                                float r = (v[q] + w[q]) * pow2f(-(le + sPhi[p * nu + a]));
                                unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(r)));
                                if (lane == 0) atomicMax(&rowmax[gl * nu + a], m);
                            }
                        }
                    }
                }
                __syncthreads();
            }
            for (int k = half; k < T; k += 2) {
                const int gl = k * GPT + g_in_tile;
                const int ge = gb * GT + gl;
                const int le = (F16 && ge < G1) ? lexp[ge] : 0;
                for (int a0 = 0; a0 < nu; a0 += 16) {
                    float v[16];
                    tc::tmem_ld16(taddr + lane_base + (uint32_t)(k * NB1 + p * nu + a0), v);
                    if (F16) {
                        float w[16];
                        tc::tmem_ld16(taddr + lane_base + (uint32_t)(c1col + k * NB1 + p * nu + a0), w);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int q = 0; q < 16; ++q) v[q] += w[q];
                    } else {
                        tc::tmem_ld_wait();
                    }
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int a = a0 + q;
                        if (a < nu) {
                            float r = v[q];
                            if (F16) r *= pow2f(row_exp(rowmax[gl * nu + a]) - le - sPhi[p * nu + a]);
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
                    const uint32_t acc = s > 0 ? 1u : 0u;
                    tc::mma_f16(d, ah, bh, id2, acc);
                    if (F16) {
                        const uint32_t dc = d + (uint32_t)NB2;
                        tc::mma_f16(dc, ah, bl, id2, acc);
                        tc::mma_f16(dc, al, bh, id2, 1u);
                        tc::mma_f16(dc, al, bl, id2, 1u);
                    } else {
                        tc::mma_f16(d, ah, bl, id2, 1u);
                        tc::mma_f16(d, al, bh, id2, 1u);
                    }
                }
                tc::mma_commit(&done_bar);
            }
            __syncwarp();
            {
                bool ok = tc::mbar_wait(&done_bar, done_phase, lim);
                done_phase ^= 1;
                if (__syncthreads_or(!ok)) { failed = true; break; }
                tc::fence_after_sync();
            }
            // epilogue 2: thread (lane r, half s) holds row r = (gbl, a) of M for spin s;
            // rows to shared memory as Ms[((gbl * 2 + s) * nu + a) * nu + b] (re, im)
            const int r = Lrow;
            const int gbl = r / nu, a = r % nu;
            const int spin = half;
            const int ns = spin ? nd : nu;
            const int cb = spin ? 2 * nu : 0;
            const bool row_ok = r < GT * nu && a < ns;
            const int er = F16 ? row_exp(rowmax[min(r, 127)]) : 0;
            for (int c0 = 0; c0 < NB2; c0 += 16) {
                if (c0 + 16 <= cb || c0 >= cb + 2 * ns) continue;   // uniform across the warp
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
                        const int c = c0 + q - cb;
                        if (c >= 0 && c < 2 * ns) {
                            const int b = c < ns ? c : c - ns, im = c >= ns;
                            float x = v[q];
                            if (F16) x *= pow2f(-(er + sTh[p * NB2 + c0 + q]));
                            Ms[2 * (((gbl * 2 + spin) * nu + a) * nu + b) + im] = x;
                        }
                    }
                }
            }
            tc::fence_before_sync();
            __syncthreads();
            {
                float2 tr = make_float2(0.f, 0.f), ex = make_float2(0.f, 0.f);
                if (row_ok) {
                    const float* Mb = Ms + 2 * ((gbl * 2 + spin) * nu * nu);
                    tr = make_float2(Mb[2 * (a * nu + a)], Mb[2 * (a * nu + a) + 1]);
                    float exx = 0.f, exy = 0.f;
                    for (int b = 0; b < ns; ++b) {
                        const float x1 = Mb[2 * (a * nu + b)], y1 = Mb[2 * (a * nu + b) + 1];
                        const float x2 = Mb[2 * (b * nu + a)], y2 = Mb[2 * (b * nu + a) + 1];
                        exx = fmaf(x1, x2, fmaf(-y1, y2, exx));
                        exy = fmaf(x1, y2, fmaf(y1, x2, exy));
                    }
                    ex = make_float2(exx, exy);
                }
                red_tr[spin][r] = tr;
                red_ex[spin][r] = ex;
            }
            __syncthreads();
            // sums over a and the spins in FP32 (FP64 is slow on this part), one
            // FP64 accumulation per pair and block of matrices
            if (tid < GT) {
                float trx = 0.f, tryy = 0.f, exx = 0.f, exy = 0.f;
                for (int sp = 0; sp < 2; ++sp)
                    for (int aa = 0; aa < nu; ++aa) {
                        const float2 x = red_tr[sp][tid * nu + aa], y = red_ex[sp][tid * nu + aa];
                        trx += x.x; tryy += x.y;
                        exx += y.x; exy += y.y;
                    }
                const int ge = gb * GT + tid;    // index into (h, L_0, L_1, ...)
                float2 c = make_float2(0.f, 0.f);
                if (ge == 0) {
                    c = make_float2(trx, tryy);
                } else if (ge <= G) {
                    vpair[(pair0 + p) * (long long)G + (ge - 1)] = cmk((double)trx, (double)tryy);
                    c = make_float2(0.5f * (trx * trx - tryy * tryy - exx), 0.5f * (2.f * trx * tryy - exy));
                }
                red_cf[tid] = c;
            }
            __syncthreads();
            if (warp == 0) {
                float cx = 0.f, cy = 0.f;
                for (int q = lane; q < GT; q += 32) { cx += red_cf[q].x; cy += red_cf[q].y; }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    cx += __shfl_xor_sync(0xffffffffu, cx, off);
                    cy += __shfl_xor_sync(0xffffffffu, cy, off);
                }
                if (lane == 0) eacc[p] = cadd(eacc[p], cmk((double)cx, (double)cy));
            }
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
        }
    }
    if (failed) {
        // drain: every issued copy and MMA completes before the block releases its memory
        if (tid == 0) {
            atomicOr(status, STATUS_TIMEOUT);
            for (int v = max(consumed, loaded - S); v < loaded; ++v)
                if (v >= 0) tc::mbar_wait(&full_bar[v % S], (uint32_t)((v / S) & 1), 1u << 22);
            tc::mma_commit(&drain_bar);
            tc::mbar_wait(&drain_bar, 0, 1u << 22);
        }
    } else if (tid < np) {
        epair[pair0 + tid] = eacc[tid];
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

// ---------------------------------------------------------------- walker-side form (N <= 64)
// With Theta_p = phi_w A_p^-1 and B_p = Phi_p A_p^-T, the matrix
// M'_g = B_p^T (X_g phi_w) = A_p^-1 M_g A_p has the traces of M_g = Phi_p^T X_g Theta_p,
// and Y_g = X_g phi_w depends on the walker only.  Two kernels:
//   tcy_y_kernel (two blocks per walker, half of its units each) forms, per
//     operand unit of two matrices,
//     GEMM-Y  D_Y[(g, j), c] = sum_i X_g[j, i] PW[c, i],  PW rows c = [Re phi | Im phi],
//     and its epilogue: the split image BY_g with rows
//       BY row (col', re) = [Re Y_g[:, col'] | -Im Y_g[:, col']],
//       BY row (col', im) = [Im Y_g[:, col'] |  Re Y_g[:, col']]   (K = 2 x 64),
//     per-matrix power-of-two scale, the two matrices' images as one operand of
//     2 NBY rows, written to global memory in the swizzled layout the MMAs read,
//     plus the scale exponents;
//   contract_tcy_kernel (one block per PG pairs of a walker) streams those
//     images through a ring of bulk copies and runs
//     GEMM-M  D_M[(p, col), (h, col', ri)] = sum_k AM[(p, col), k] BY_g+h[(col', ri), k],
//     AM row (p, col) = [Re B_p[:, col] | Im B_p[:, col]], so
//     D_M[(p, col), (h, col', re/im)] = Re/Im (B_p^T Y_g+h)[col, col'] (same-spin blocks
//     used), one MMA per K step and product for both matrices; a producer warp
//     issues copies and MMAs into two tensor-memory buffers while the other eight
//     warps run epilogue M (shared-memory transpose, traces, sums) on the other,
//     the two halves of them on the two matrices of a unit.
// So the image of Y_g, whose epilogue dominated the fused kernel, is formed once
// per walker instead of once per block of pairs.
constexpr int TCY_MAXPG = 64;

__host__ __device__ __forceinline__ size_t tcy_unit_bytes(int NBY) { return 4 * (size_t)NBY * 128 * 2; }

template <bool F16>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tcy_y_kernel(int N, int nu, int nd, int G, int NBY, int S, int parts, const uint8_t* __restrict__ image,
                 const int* __restrict__ lexp, const double2* __restrict__ phi, uint8_t* __restrict__ yimg,
                 int* __restrict__ yexp, int* status, uint32_t lim) {
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const int nt = nu + nd;
    uint8_t* XR = sm;                                          // S units of the (h, L_g) image
    uint8_t* PWh = XR + (size_t)S * TC_UNIT;                   // NBY rows x 64 K
    const size_t pw_bytes = (size_t)NBY * 64 * 2;
    uint8_t* PWl = PWh + pw_bytes;
    uint8_t* BY = PWl + pw_bytes;                              // staging: matrix h hi at 2h*by, lo at (2h+1)*by
    const size_t by_bytes = (size_t)NBY * 128 * 2;
    const size_t unit_bytes = 4 * by_bytes;
    __shared__ uint64_t full_bar[TC_MAXSTAGES], empty_bar[TC_MAXSTAGES], ybar, drain_bar;
    __shared__ uint32_t tslot;
    __shared__ int fail_flag;
    __shared__ unsigned ymax[2][2];
    __shared__ int sPW[128];
    __shared__ float cmul_pw[128];          // 2^-sPW: removes the PW row scales from D_Y

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const long long w = blockIdx.x / parts;   // walker; its units are split over `parts` blocks
    const int G1 = G + 1;
    const int n_units = (G1 + 1) / 2;
    const int upp = (n_units + parts - 1) / parts;
    const int u0 = (int)(blockIdx.x % parts) * upp;
    const int nloc = max(0, min(n_units, u0 + upp) - u0);   // units of this block: u0 .. u0 + nloc - 1
    const double2* phw = phi + w * (long long)N * nt;
    uint8_t* yout = yimg + (size_t)w * n_units * unit_bytes;
    int* yex = yexp + (size_t)w * 2 * n_units;

    if (warp == 0) {
        tc::tmem_alloc(&tslot, 256);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            tc::mbar_init(&full_bar[q], 1);
            tc::mbar_init(&empty_bar[q], 1);
        }
        tc::mbar_init(&ybar, 1);
        tc::mbar_init(&drain_bar, 1);
        tc::mbar_fence_init();
        fail_flag = 0;
        ymax[0][0] = ymax[0][1] = ymax[1][0] = ymax[1][1] = 0u;
    }
    // exponents of the PW rows (walker columns)
    for (int c = tid; c < 128; c += TC_THREADS) {
        float m = 0.f;
        if (F16 && c < 2 * nt) {
            const int col = c % nt, im = c >= nt;
            for (int i = 0; i < N; ++i) {
                const double2 t = phw[(long long)i * nt + col];
                m = fmaxf(m, (float)fabs(im ? t.y : t.x));
            }
        }
        sPW[c] = scale_exp<F16>(m);
        cmul_pw[c] = pow2f(-sPW[c]);
    }
    __syncthreads();
    int loaded = 0, consumed = 0;   // meaningful in thread 0
    if (tid == 0) {
        for (; loaded < S && loaded < nloc; ++loaded) {
            tc::mbar_arrive_expect_tx(&full_bar[loaded], TC_UNIT);
            tc::bulk_g2s(XR + (size_t)loaded * TC_UNIT, image + (size_t)(u0 + loaded) * TC_UNIT, TC_UNIT,
                         &full_bar[loaded]);
        }
    }
    // PW: rows c = [Re phi_w | Im phi_w] (column c), K = i
    for (int e = tid; e < NBY * 64; e += TC_THREADS) {
        const int c = e / 64, i = e % 64;
        float x = 0.f;
        if (c < 2 * nt && i < N) {
            const double2 t = phw[(long long)i * nt + (c % nt)];
            x = (float)(c >= nt ? t.y : t.x) * pow2f(sPW[c]);
        }
        split16<F16>(x, PWh, PWl, tc::sw128_offset(NBY, c, i));
    }
    // BY starts zero (rows past 2 nt are never written)
    for (int e = tid; e < (int)(unit_bytes / 16); e += TC_THREADS) reinterpret_cast<uint4*>(BY)[e] = make_uint4(0, 0, 0, 0);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    const uint32_t taddr = tslot;
    const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
    const uint32_t idd = F16 ? tc::idesc_f16_f32(128, NBY) : tc::idesc_bf16_f32(128, NBY);
    const uint32_t dyc = F16 ? (uint32_t)NBY : 0u;                  // correction columns of D_Y
    const int Lrow = 32 * quarter + lane;
    uint32_t y_ph = 0;
    bool failed = false;

    auto refill_upto = [&](int last_consumed) -> bool {
        while (loaded < nloc && loaded - S <= last_consumed) {
            const int v = loaded - S, st = loaded % S;
            if (v >= 0 && !tc::mbar_wait(&empty_bar[st], (uint32_t)((v / S) & 1), lim)) return false;
            tc::mbar_arrive_expect_tx(&full_bar[st], TC_UNIT);
            tc::bulk_g2s(XR + (size_t)st * TC_UNIT, image + (size_t)(u0 + loaded) * TC_UNIT, TC_UNIT, &full_bar[st]);
            ++loaded;
        }
        return true;
    };
    // GEMM-Y of this block's unit u (local index; thread 0): D_Y = X(unit) PW^T
    auto issue_Y = [&](int u) -> bool {
        const int st = u % S;
        if (!tc::mbar_wait(&full_bar[st], (uint32_t)((u / S) & 1), lim)) return false;
        tc::fence_after_sync();
        const uint32_t sa = tc::smem_u32(XR + (size_t)st * TC_UNIT);
#pragma unroll
        for (int ss = 0; ss < 4; ++ss) {
            const uint64_t ah = tc::desc_sw128(sa + ss * 32), al = tc::desc_sw128(sa + 16384 + ss * 32);
            const uint64_t bh = tc::desc_sw128(tc::smem_u32(PWh) + ss * 32), bl = tc::desc_sw128(tc::smem_u32(PWl) + ss * 32);
            const uint32_t acc = ss > 0 ? 1u : 0u;
            tc::mma_f16(taddr, ah, bh, idd, acc);
            if (F16) {
                tc::mma_f16(taddr + dyc, ah, bl, idd, acc);
                tc::mma_f16(taddr + dyc, al, bh, idd, 1u);
                tc::mma_f16(taddr + dyc, al, bl, idd, 1u);
            } else {
                tc::mma_f16(taddr, ah, bl, idd, 1u);
                tc::mma_f16(taddr, al, bh, idd, 1u);
            }
        }
        tc::mma_commit(&empty_bar[st]);
        tc::mma_commit(&ybar);
        ++consumed;
        return refill_upto(u - 1);
    };
    if (tid == 0 && nloc > 0 && !issue_Y(0)) fail_flag = 1;

    const int gi = Lrow / 64, jrow = Lrow % 64;      // D_Y row: matrix in unit, j
    const int ch = (nt + 1) / 2;                      // walker columns per half
    const int cl = half * ch, cn = min(nt, cl + ch) - cl;
    for (int v = 0; v < nloc && !failed; ++v) {
        const int u = u0 + v;   // unit of the walker's image
        __syncwarp();
        {
            bool ok = fail_flag == 0 && tc::mbar_wait(&ybar, y_ph, lim);
            y_ph ^= 1;
            if (__syncthreads_or(!ok || fail_flag)) { failed = true; break; }
            tc::fence_after_sync();
        }
        if (tid == 0) ymax[(u + 1) & 1][0] = ymax[(u + 1) & 1][1] = 0u;
        // ---- epilogue Y: Y_g[j, col] for this thread's columns (two passes over
        // tensor memory: the matrix maximum, then scaled, split and stored in BY_g)
        {
            const int g = 2 * u + gi;
            const int le = (F16 && g < G1) ? lexp[g] : 0;
            // one image of 2 NBY rows for the unit's two matrices (matrix gi from row gi NBY),
            // so the pair kernel multiplies both with one MMA per K step and product
            uint8_t* byh = BY + (size_t)gi * NBY * 128;
            uint8_t* byl = BY + 2 * by_bytes + (size_t)gi * NBY * 128;
            // K position jrow of a BY row: within a 128-byte row, chunk (jrow / 8) xor (row % 8)
            const uint32_t kb1 = 2u * (uint32_t)NBY * 128u;     // second K block (k = 64 + jrow)
            float mul = pow2f(-le);
            for (int pass = F16 ? 0 : 1; pass < 2; ++pass) {
                float mx = 0.f;
                for (int c0 = 0; c0 < ch; c0 += 16) {   // uniform across the block
                    float v[16], vi[16];
                    tc::tmem_ld16(taddr + lane_base + (uint32_t)(cl + c0), v);
                    tc::tmem_ld16(taddr + lane_base + (uint32_t)(nt + cl + c0), vi);
                    if (F16) {
                        float vc[16], vic[16];
                        tc::tmem_ld16(taddr + lane_base + dyc + (uint32_t)(cl + c0), vc);
                        tc::tmem_ld16(taddr + lane_base + dyc + (uint32_t)(nt + cl + c0), vic);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int q = 0; q < 16; ++q) { v[q] += vc[q]; vi[q] += vic[q]; }
                    } else {
                        tc::tmem_ld_wait();
                    }
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int idx = c0 + q, col = cl + idx;
                        if (idx < cn) {
                            const float a = v[q] * (mul * cmul_pw[col]);
                            const float b = vi[q] * (mul * cmul_pw[nt + col]);
                            if (pass == 0) {
                                mx = fmaxf(mx, fmaxf(fabsf(a), fabsf(b)));
                            } else {
                                uint16_t xh, xl, yh, yl;
                                split_bits<F16>(a, xh, xl);
                                split_bits<F16>(b, yh, yl);
                                const int n0 = 2 * col, n1 = n0 + 1;   // rows (col, re), (col, im)
                                const uint32_t o0 = (uint32_t)(n0 >> 3) * 1024u + (uint32_t)(n0 & 7) * 128u +
                                                    (uint32_t)(((jrow >> 3) ^ (n0 & 7)) * 16 + (jrow & 7) * 2);
                                const uint32_t o1 = (uint32_t)(n1 >> 3) * 1024u + (uint32_t)(n1 & 7) * 128u +
                                                    (uint32_t)(((jrow >> 3) ^ (n1 & 7)) * 16 + (jrow & 7) * 2);
                                // row (col, re) = [Re Y | -Im Y], row (col, im) = [Im Y | Re Y]
                                *reinterpret_cast<uint16_t*>(byh + o0) = xh;
                                *reinterpret_cast<uint16_t*>(byl + o0) = xl;
                                *reinterpret_cast<uint16_t*>(byh + o0 + kb1) = yh ^ 0x8000u;
                                *reinterpret_cast<uint16_t*>(byl + o0 + kb1) = yl ^ 0x8000u;
                                *reinterpret_cast<uint16_t*>(byh + o1) = yh;
                                *reinterpret_cast<uint16_t*>(byl + o1) = yl;
                                *reinterpret_cast<uint16_t*>(byh + o1 + kb1) = xh;
                                *reinterpret_cast<uint16_t*>(byl + o1 + kb1) = xl;
                            }
                        }
                    }
                }
                if (pass == 0) {
                    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
                    if (lane == 0) atomicMax(&ymax[u & 1][gi], m);
                    __syncthreads();
                    mul *= pow2f(row_exp(ymax[u & 1][gi]));
                }
            }
        }
        // D_Y is read; the next unit's GEMM-Y overlaps the copy of this unit's image
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            yex[2 * u] = F16 ? row_exp(ymax[u & 1][0]) : 0;
            yex[2 * u + 1] = F16 ? row_exp(ymax[u & 1][1]) : 0;
            if (v + 1 < nloc && !issue_Y(v + 1)) fail_flag = 1;
        }
        const uint4* src = reinterpret_cast<const uint4*>(BY);
        uint4* dst = reinterpret_cast<uint4*>(yout + (size_t)u * unit_bytes);
        for (int e = tid; e < (int)(unit_bytes / 16); e += TC_THREADS) dst[e] = src[e];
        __syncthreads();   // the staging area is free for the next epilogue
    }
    if (failed && tid == 0) {
        // drain: every issued copy and MMA completes before the block releases its memory
        atomicOr(status, STATUS_TIMEOUT);
        for (int v = max(consumed, loaded - S); v < loaded; ++v)
            if (v >= 0) tc::mbar_wait(&full_bar[v % S], (uint32_t)((v / S) & 1), 1u << 22);
        tc::mma_commit(&drain_bar);
        tc::mbar_wait(&drain_bar, 0, 1u << 22);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 256);
}

// Pair kernel: warps 0-7 run epilogue M (two halves, one matrix of the unit
// each; they synchronise on named barrier 1), warp 8 is the producer: it streams
// the Y images into the ring, waits for a D_M buffer to be free, and issues
// GEMM-M.  mbarriers: full_bar (a unit's image has landed), empty_bar (the MMAs
// reading a ring stage have completed), mfull (GEMM-M of a unit has completed),
// mempty (the epilogue has read a D_M buffer).  nbuf: D_M buffers (2 when both
// fit in tensor memory).  Every wait is bounded; on a timeout the warps stop,
// the producer drains its copies and MMAs, and the block returns.
constexpr int TCY_THREADS = TC_THREADS + 32;

template <bool F16>
__global__ void __launch_bounds__(TCY_THREADS, 1)
    contract_tcy_kernel(int N, int nu, int nd, int G, int P, int PG, int NBY, int S, int nbuf,
                        const uint8_t* __restrict__ yimg, const int* __restrict__ yexp,
                        const double2* __restrict__ Bm, double2* __restrict__ vpair, double2* __restrict__ epair,
                        int* status, uint32_t lim) {
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const int nt = nu + nd;
    const int S2 = nu * nu + nd * nd;
    const size_t by_bytes = (size_t)NBY * 128 * 2;
    const uint32_t unit_bytes = (uint32_t)(4 * by_bytes);
    uint8_t* YR = sm;                                          // S units of the Y images
    uint8_t* AMh = YR + (size_t)S * unit_bytes;                // 128 rows x 128 K
    uint8_t* AMl = AMh + 128 * 128 * 2;
    float* Ms = reinterpret_cast<float*>(AMl + 128 * 128 * 2);  // matrix h: PG x S2 complex
    __shared__ uint64_t full_bar[TC_MAXSTAGES], empty_bar[TC_MAXSTAGES], mfull[2], mempty[2], drain_bar;
    __shared__ uint32_t tslot;
    __shared__ float2 red_tr[2][128], red_ex[2][128];
    __shared__ double2 eacc[2][TCY_MAXPG];
    __shared__ int sA[128];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = (warp >> 2) & 1;
    const int bpw = (P + PG - 1) / PG;
    const long long w = blockIdx.x / bpw;
    const int p0 = (int)(blockIdx.x % bpw) * PG;
    const int np = min(PG, P - p0);
    const long long pairbase = w * P + p0;
    const int G1 = G + 1;
    const int n_units = (G1 + 1) / 2;
    const uint8_t* ysrc = yimg + (size_t)w * n_units * unit_bytes;
    const int* yex = yexp + (size_t)w * 2 * n_units;

    if (warp == 0) {
        tc::tmem_alloc(&tslot, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            tc::mbar_init(&full_bar[q], 1);
            tc::mbar_init(&empty_bar[q], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&mfull[b], 1);
            tc::mbar_init(&mempty[b], 1);
        }
        tc::mbar_init(&drain_bar, 1);
        tc::mbar_fence_init();
    }
    if (tid < 2 * TCY_MAXPG) eacc[tid / TCY_MAXPG][tid % TCY_MAXPG] = cmk(0.0, 0.0);
    // exponents of the AM rows (B columns)
    for (int r = tid; r < 128; r += TCY_THREADS) {
        const int p = r / nt, col = r % nt;
        float m = 0.f;
        if (F16 && p < np) {
            const double2* Bp = Bm + (pairbase + p) * (long long)N * nt;
            for (int j = 0; j < N; ++j) {
                const double2 t = Bp[(long long)j * nt + col];
                m = fmaxf(m, fmaxf((float)fabs(t.x), (float)fabs(t.y)));
            }
        }
        sA[r] = scale_exp<F16>(m);
    }
    __syncthreads();
    // AM: row (p, col) = [Re B_p[:, col] | Im B_p[:, col]]
    for (int e = tid; e < 128 * 128; e += TCY_THREADS) {
        const int r = e / 128, k = e % 128;
        const int j = k & 63, ri = k >> 6;
        const int p = r / nt, col = r % nt;
        float x = 0.f;
        if (p < np && j < N) {
            const double2 t = Bm[(pairbase + p) * (long long)N * nt + (long long)j * nt + col];
            x = (float)(ri ? t.y : t.x) * pow2f(sA[r]);
        }
        split16<F16>(x, AMh, AMl, tc::sw128_offset(128, r, k));
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    const uint32_t taddr = tslot;
    const uint32_t idd = F16 ? tc::idesc_f16_f32(128, 2 * NBY) : tc::idesc_bf16_f32(128, 2 * NBY);
    const uint32_t dms = F16 ? 2u * NBY : (uint32_t)NBY;            // columns of one matrix's D_M
    bool failed = false;

    if (warp == 8) {
        // ---- producer (one thread)
        if (lane == 0) {
            int loaded = 0, consumed = 0;
            auto load = [&](int st, int v) {
                tc::mbar_arrive_expect_tx(&full_bar[st], unit_bytes);
                tc::bulk_g2s(YR + (size_t)st * unit_bytes, ysrc + (size_t)v * unit_bytes, unit_bytes, &full_bar[st]);
            };
            for (; loaded < S && loaded < n_units; ++loaded) load(loaded, loaded);
            for (int u = 0; u < n_units && !failed; ++u) {
                const int b = u % nbuf, st = u % S;
                // unit u not loaded yet (a one-stage ring): its stage frees when GEMM-M of unit u - S completes
                while (loaded <= u) {
                    const int v = loaded - S, sv = loaded % S;
                    if (v >= 0 && !tc::mbar_wait(&empty_bar[sv], (uint32_t)((v / S) & 1), lim)) { failed = true; break; }
                    load(sv, loaded);
                    ++loaded;
                }
                if (failed) break;
                // D_M buffer b is free once the epilogue of unit u - nbuf has read it
                if (u >= nbuf && !tc::mbar_wait(&mempty[b], (uint32_t)((u / nbuf - 1) & 1), lim)) { failed = true; break; }
                if (!tc::mbar_wait(&full_bar[st], (uint32_t)((u / S) & 1), lim)) { failed = true; break; }
                tc::fence_after_sync();
                ++consumed;
                // both matrices of the unit in one operand of 2 NBY rows; D columns of buffer b:
                // [matrix 0 | matrix 1] then (FP16) their corrections
                const uint8_t* byh = YR + (size_t)st * unit_bytes;
                const uint8_t* byl = byh + 2 * by_bytes;
                const uint32_t d = taddr + (uint32_t)b * 2u * dms;
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const uint32_t ka = (uint32_t)((s >> 2) * 128 * 128 + (s & 3) * 32);
                    const uint32_t kbo = (uint32_t)((s >> 2) * 2 * NBY * 128 + (s & 3) * 32);
                    const uint64_t ah = tc::desc_sw128(tc::smem_u32(AMh) + ka),
                                   al = tc::desc_sw128(tc::smem_u32(AMl) + ka);
                    const uint64_t bh = tc::desc_sw128(tc::smem_u32(byh) + kbo),
                                   bl = tc::desc_sw128(tc::smem_u32(byl) + kbo);
                    const uint32_t acc = s > 0 ? 1u : 0u;
                    tc::mma_f16(d, ah, bh, idd, acc);
                    if (F16) {
                        tc::mma_f16(d + 2u * NBY, ah, bl, idd, acc);
                        tc::mma_f16(d + 2u * NBY, al, bh, idd, 1u);
                        tc::mma_f16(d + 2u * NBY, al, bl, idd, 1u);
                    } else {
                        tc::mma_f16(d, ah, bl, idd, 1u);
                        tc::mma_f16(d, al, bh, idd, 1u);
                    }
                }
                tc::mma_commit(&empty_bar[st]);
                tc::mma_commit(&mfull[b]);
                // refill the stages whose MMAs (units up to u - 1) have completed
                while (loaded < n_units && loaded - S <= u - 1) {
                    const int v = loaded - S, sv = loaded % S;
                    if (!tc::mbar_wait(&empty_bar[sv], (uint32_t)((v / S) & 1), lim)) { failed = true; break; }
                    load(sv, loaded);
                    ++loaded;
                }
            }
            if (failed) {
                atomicOr(status, STATUS_TIMEOUT);
            }
            // drain: every issued copy and MMA completes before the block releases its memory
            for (int v = max(consumed, loaded - S); v < loaded; ++v)
                if (v >= 0) tc::mbar_wait(&full_bar[v % S], (uint32_t)((v / S) & 1), 1u << 22);
            tc::mma_commit(&drain_bar);
            tc::mbar_wait(&drain_bar, 0, 1u << 22);
        }
        __syncwarp();
    } else {
        // ---- epilogue warps 0-7
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        const int Lrow = 32 * quarter + lane;
        uint32_t m_ph0 = 0, m_ph1 = 0;
        for (int u = 0; u < n_units; ++u) {
            const int b = u % nbuf;
            const bool ok = tc::mbar_wait(&mfull[b], b ? m_ph1 : m_ph0, lim);
            if (b) m_ph1 ^= 1; else m_ph0 ^= 1;
            if (tc::named_sync_or<TC_THREADS>(!ok)) { failed = true; break; }
            tc::fence_after_sync();
        // ---- epilogue M: half h takes matrix 2u + h; thread lane r = (p, col)
        {
            const int r = Lrow;
            const int p = r / nt, col = r % nt;
            const int spin = col < nu ? 0 : 1;
            const int a = spin ? col - nu : col;
            const int off = spin ? nu : 0, ns = spin ? nd : nu;
            const bool row_ok = p < np;
            const float sc = F16 ? pow2f(-(sA[r] + yex[2 * u + half])) : 1.f;
            const uint32_t dcol = (uint32_t)(u % nbuf) * 2u * dms + (uint32_t)half * NBY;
            float* Mg = Ms + (size_t)half * PG * S2 * 2;
            float* Mrow = Mg + 2 * ((size_t)p * S2 + (spin ? nu * nu : 0));
            for (int c0 = 0; c0 < 2 * nt; c0 += 16) {
                float v[16];
                tc::tmem_ld16(taddr + lane_base + dcol + (uint32_t)c0, v);
                if (F16) {
                    float vc[16];
                    tc::tmem_ld16(taddr + lane_base + dcol + 2u * (uint32_t)NBY + (uint32_t)c0, vc);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] += vc[q];
                } else {
                    tc::tmem_ld_wait();
                }
                if (row_ok) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int n = c0 + q, cp = n >> 1;
                        if (cp >= off && cp < off + ns) Mrow[2 * (a * ns + (cp - off)) + (n & 1)] = v[q] * sc;
                    }
                }
            }
            tc::fence_before_sync();
            tc::named_sync<TC_THREADS>();
            float2 tr = make_float2(0.f, 0.f), ex = make_float2(0.f, 0.f);
            if (row_ok) {
                tr = make_float2(Mrow[2 * (a * ns + a)], Mrow[2 * (a * ns + a) + 1]);
                float exx = 0.f, exy = 0.f;
                for (int b = 0; b < ns; ++b) {
                    const float x1 = Mrow[2 * (a * ns + b)], y1 = Mrow[2 * (a * ns + b) + 1];
                    const float x2 = Mrow[2 * (b * ns + a)], y2 = Mrow[2 * (b * ns + a) + 1];
                    exx = fmaf(x1, x2, fmaf(-y1, y2, exx));
                    exy = fmaf(x1, y2, fmaf(y1, x2, exy));
                }
                ex = make_float2(exx, exy);
            }
            red_tr[half][r] = tr;
            red_ex[half][r] = ex;
            tc::named_sync<TC_THREADS>();
            // per pair: sums over its rows in FP32 (FP64 is slow on this part), the
            // energy term of the matrix, then one FP64 accumulation per pair and unit
            // lpp consecutive threads (one warp) share the rows of a pair, then combine by shuffles
            {
                const int lpp = 8 * PG <= TC_THREADS ? 4 : (4 * PG <= TC_THREADS ? 2 : 1);
                const int slot = tid / lpp, q = tid % lpp;
                const int hh = slot / PG, pp = slot % PG;
                const bool mine = slot < 2 * PG && pp < np;
                float trx = 0.f, tryy = 0.f, exx = 0.f, exy = 0.f;
                if (mine) {
                    const float2* rt = &red_tr[hh][pp * nt];
                    const float2* re = &red_ex[hh][pp * nt];
                    for (int cc = q; cc < nt; cc += lpp) {
                        const float2 x = rt[cc], y = re[cc];
                        trx += x.x; tryy += x.y;
                        exx += y.x; exy += y.y;
                    }
                }
                for (int o = 1; o < lpp; o <<= 1) {   // every epilogue thread takes part
                    trx += __shfl_xor_sync(0xffffffffu, trx, o);
                    tryy += __shfl_xor_sync(0xffffffffu, tryy, o);
                    exx += __shfl_xor_sync(0xffffffffu, exx, o);
                    exy += __shfl_xor_sync(0xffffffffu, exy, o);
                }
                if (mine && q == 0) {
                    float2 c = make_float2(0.f, 0.f);
                    const int ge = 2 * u + hh;    // index into (h, L_0, L_1, ...)
                    if (ge == 0) {
                        c = make_float2(trx, tryy);
                    } else if (ge <= G) {
                        vpair[(pairbase + pp) * (long long)G + (ge - 1)] = cmk((double)trx, (double)tryy);
                        c = make_float2(0.5f * (trx * trx - tryy * tryy - exx), 0.5f * (2.f * trx * tryy - exy));
                    }
                    eacc[hh][pp] = cadd(eacc[hh][pp], cmk((double)c.x, (double)c.y));   // one thread per slot
                }
            }
            tc::fence_before_sync();
            tc::named_sync<TC_THREADS>();
            tc::fence_after_sync();
        }
            if (tid == 0) tc::mbar_arrive(&mempty[b]);   // D_M buffer b has been read
        }
        if (failed && tid == 0) atomicOr(status, STATUS_TIMEOUT);
        if (!failed && tid < np) epair[pairbase + tid] = cadd(eacc[0][tid], eacc[1][tid]);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

struct TcyShape {
    int PG, NBY, S, SY, nbuf;
    size_t smem, smem_y;
};

static size_t tcy_smem_bytes(int nu, int nd, int PG, int NBY, int S) {
    return 1024 + (size_t)S * tcy_unit_bytes(NBY) + 2 * (size_t)128 * 128 * 2 +
           2 * (size_t)PG * (nu * nu + nd * nd) * 8;
}

static size_t tcy_y_smem_bytes(int NBY, int S) {
    return 1024 + (size_t)S * TC_UNIT + 2 * (size_t)NBY * 64 * 2 + tcy_unit_bytes(NBY);
}

// Shape of the walker-side form: N <= 64, n_up + n_dn <= 40, PG pairs per block
// with PG (n_up + n_dn) <= 128 rows of AM.  Tensor memory: D_Y of the image
// kernel (NBY columns, doubled for the FP16 corrections) in 256 columns; D_M of
// the pair kernel (two matrices, NBY columns each plus as many corrections) once
// or, when it fits the 512 columns, twice.
static bool tcy_shape(int N, int nu, int nd, bool f16, int pg_override, TcyShape& s) {
    const int nt = nu + nd;
    if (N < 1 || N > 64 || nu < 1 || nd < 0 || nd > nu || nt > 40) return false;
    s.NBY = ((2 * nt + 15) / 16) * 16;
    const int dm = (f16 ? 2 : 1) * s.NBY;          // D_M columns of one matrix
    if ((f16 ? 2 : 1) * s.NBY > 256 || 2 * dm > 512) return false;
    s.nbuf = 4 * dm <= 512 ? 2 : 1;
    s.PG = min(TCY_MAXPG, 128 / nt);
    if (pg_override > 0 && pg_override < s.PG) s.PG = pg_override;
    for (s.S = TC_MAXSTAGES; s.S >= 1; --s.S) {
        s.smem = tcy_smem_bytes(nu, nd, s.PG, s.NBY, s.S);
        if (s.smem <= TC_SMEM_MAX) break;
    }
    if (s.S < 1) return false;
    for (s.SY = TC_MAXSTAGES; s.SY >= 2; --s.SY) {
        s.smem_y = tcy_y_smem_bytes(s.NBY, s.SY);
        if (s.smem_y <= TC_SMEM_MAX) return true;
    }
    return false;
}

bool contract_tc_walker_side(int N, int nu, int nd, bool f16) {
    TcyShape s;
    return tcy_shape(N, nu, nd, f16, 0, s);
}

size_t contract_tcy_yimage_bytes(int N, int nu, int nd, int G, long long W, bool f16) {
    TcyShape s;
    if (!tcy_shape(N, nu, nd, f16, 0, s)) return 0;
    const long long n_units = (G + 2) / 2;
    const size_t img = (size_t)W * n_units * tcy_unit_bytes(s.NBY);
    return img + (size_t)W * 2 * n_units * sizeof(int);
}

template <bool F16>
static cudaError_t launch_tcy(cudaStream_t st, const Dims& d, const TcyShape& s, const void* image, const int* lexp,
                              const double2* Bm, const double2* phi, void* ywork, double2* vpair, double2* epair,
                              int* status) {
    const long long W = d.pairs / d.P;
    const long long n_units = (d.G + 2) / 2;
    uint8_t* yimg = static_cast<uint8_t*>(ywork);
    int* yexp = reinterpret_cast<int*>(yimg + (size_t)W * n_units * tcy_unit_bytes(s.NBY));
    cudaError_t e = raise_smem_limit((const void*)tcy_y_kernel<F16>, s.smem_y);
    if (e != cudaSuccess) return e;
    // each walker's units over two blocks: twice the blocks fill the last wave better
    const int parts = n_units >= 2 ? 2 : 1;
    tcy_y_kernel<F16><<<(unsigned)(W * parts), TC_THREADS, s.smem_y, st>>>(d.N, d.nu, d.nd, d.G, s.NBY, s.SY, parts,
                                                                           (const uint8_t*)image, lexp, phi, yimg,
                                                                           yexp, status, d.wait_polls);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = raise_smem_limit((const void*)contract_tcy_kernel<F16>, s.smem);
    if (e != cudaSuccess) return e;
    const long long blocks = W * ((d.P + s.PG - 1) / s.PG);
    contract_tcy_kernel<F16><<<(unsigned)blocks, TCY_THREADS, s.smem, st>>>(d.N, d.nu, d.nd, d.G, d.P, s.PG, s.NBY, s.S,
                                                                         s.nbuf, yimg, yexp, Bm, vpair, epair, status,
                                                                         d.wait_polls);
    count_launches(1);
    return cudaGetLastError();
}

static size_t tc_smem_bytes(int NPAD, int NB1, int NB2, int TP, int S) {
    return 1024 + (size_t)S * TC_UNIT + 2 * (size_t)128 * NPAD * 2 + 2 * (size_t)NB1 * NPAD * 2 +
           2 * (size_t)TP * NB2 * NPAD * 2;
}

// Fill in TP-dependent fields; false if they do not fit.
static bool tc_fit(TcShape& s, int nu, int tp, bool f16) {
    const int nb1 = ((tp * nu + 15) / 16) * 16;
    if (nb1 > 256) return false;
    const int c1 = s.T * nb1;
    const int d2 = f16 ? 2 * c1 : c1;
    const int end = d2 + (f16 ? 2 * s.NB2 : s.NB2);
    if (end > 512) return false;
    if (tp * s.NB2 > TC_MAXSCALE_B2) return false;
    int S = TC_MAXSTAGES;
    while (S >= 2 && tc_smem_bytes(s.NPAD, nb1, s.NB2, tp, S) > TC_SMEM_MAX) --S;
    if (S < 2) return false;
    s.TP = tp;
    s.NB1 = nb1;
    s.c1col = c1;
    s.d2col = d2;
    s.S = S;
    s.smem = tc_smem_bytes(s.NPAD, nb1, s.NB2, tp, S);
    return true;
}

// Tile shape for (N, n_up, n_dn): the deepest stack of matrices in GEMM2
// (GT * n_up <= 128 rows) and then the most pairs per block (TP) that fit
// tensor memory and shared memory.  Tensor-memory columns, in order: T = GT/GPT
// D1 tiles of NB1, (FP16 mode) their T correction tiles, D2 of NB2, (FP16 mode)
// its correction of NB2.  Shared memory: S >= 2 ring stages of one 32 KB unit,
// A2 (also the epilogue-2 staging), B1, and B2 of the TP pairs.
static bool tc_shape(int N, int nu, int nd, bool f16, TcShape& s) {
    s.NPAD = N <= 64 ? 64 : (N <= 128 ? 128 : 0);
    if (!s.NPAD || nu < 1 || nu > 32 || nd > nu || nd < 0) return false;
    s.GPT = 128 / s.NPAD;
    s.NKB = s.NPAD / 64;
    s.NB2 = ((2 * (nu + nd) + 15) / 16) * 16;
    for (int gt = (128 / nu) / s.GPT * s.GPT; gt >= s.GPT; gt -= s.GPT) {
        const size_t ms = (size_t)gt * 2 * nu * nu * 8;
        if (ms > 2 * (size_t)128 * s.NPAD * 2) continue;
        s.GT = gt;
        s.T = gt / s.GPT;
        for (int tp = TC_MAXTP; tp >= 1; --tp)
            if (tc_fit(s, nu, tp, f16)) return true;
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
    return (size_t)tiles * s.NKB * TC_UNIT + (size_t)G1p * sizeof(int);
}

// The split image of (h, L_g) and, after it, the per-matrix exponents.
cudaError_t contract_tc_prepare(cudaStream_t st, int N, int nu, int nd, int G, const double* h, const double* L,
                                void* image, bool f16) {
    TcShape s;
    if (!tc_shape(N, nu, nd, f16, s)) return cudaErrorInvalidValue;
    long long G1p = (long long)((G + 1 + s.GT - 1) / s.GT) * s.GT;
    int tiles = (int)(G1p / s.GPT);
    int* lexp = reinterpret_cast<int*>(static_cast<uint8_t*>(image) + (size_t)tiles * s.NKB * TC_UNIT);
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
        d.N, d.nu, d.nd, d.G, s.TP, s.GT, s.NB1, s.NB2, s.S, s.c1col, s.d2col, d.pairs, (const uint8_t*)image, lexp, Phi,
        Theta, vpair, epair, status, d.wait_polls); count_launches(1);
    return cudaGetLastError();
}

cudaError_t contract_tc(cudaStream_t st, const Dims& d, const void* image, const double* Phi, const double2* Theta,
                        const double2* phi, void* ywork, double2* vpair, double2* epair, int* status, bool f16) {
    TcShape s;
    if (!tc_shape(d.N, d.nu, d.nd, f16, s)) return cudaErrorInvalidValue;
    if (d.pairs <= 0) return cudaSuccess;
    long long G1p = (long long)((d.G + 1 + s.GT - 1) / s.GT) * s.GT;
    const int* lexp = reinterpret_cast<const int*>(static_cast<const uint8_t*>(image) +
                                                   (size_t)(G1p / s.GPT) * s.NKB * TC_UNIT);
    TcyShape sy;
    if (ywork && tcy_shape(d.N, d.nu, d.nd, f16, d.tc_tp, sy)) {   // Theta holds B = Phi A^-T here
        if (d.P < 1 || d.pairs % d.P != 0) return cudaErrorInvalidValue;
        return f16 ? launch_tcy<true>(st, d, sy, image, lexp, Theta, phi, ywork, vpair, epair, status)
                   : launch_tcy<false>(st, d, sy, image, lexp, Theta, phi, ywork, vpair, epair, status);
    }
    if (d.tc_tp > 0 && d.tc_tp < s.TP && !tc_fit(s, d.nu, d.tc_tp, f16)) return cudaErrorInvalidValue;
    if (s.NPAD == 64)
        return f16 ? launch_tc<64, true>(st, d, s, image, lexp, Phi, Theta, vpair, epair, status)
                   : launch_tc<64, false>(st, d, s, image, lexp, Phi, Theta, vpair, epair, status);
    return f16 ? launch_tc<128, true>(st, d, s, image, lexp, Phi, Theta, vpair, epair, status)
               : launch_tc<128, false>(st, d, s, image, lexp, Phi, Theta, vpair, epair, status);
}

}  // namespace afq
