// The proposal matrices S_p = sum_k x'_pk U_k of every Metropolis proposal (the
// argument of exp(S) Phi0 in Eq. (20)-(21)) on the tensor cores, for the mixed
// path's tensor-core trial orbitals (trial_tc.cu), whose digits of S' carry the
// same precision.
//
// S[p, e] = sum_k X[p, k] U[k, e] (e = the N^2 entries of S, K <= 128 variables)
// with both operands split error-free into five 8-bit digits (digits.cuh): X row
// p scaled by 2^erow[p], U column e by 2^fU[e], so that each lies in [128, 256)
// at its largest.  The A operand is U (128 columns e per tile, K-major), whose
// digit images are formed once when the context starts (sprop_u_images); the B
// operand is the digits of a block's 48 proposals side by side (rows j 48 + p,
// digit j), formed by the block itself.  One MMA of digit i of U against the
// digits 0 .. 4 - i of X adds U_i X_j to accumulator i + j for every j; the
// orders 0 .. 4 (15 digit products) are kept, every partial sum is an integer
// below (2 * 256 * 129 + 3 * 129^2) * 128 < 2^24 (exact in FP32), and an entry's
// error is about 2^-38 of K max_k |x_pk| max_k |U_k[e]|.
//
// Block: 48 proposals, persistent over the column tiles of S (320 threads): warp 0
// streams U's digit tiles (16 KB each: digit i, K block kb, 128 columns) through a
// ring of bulk copies, warp 1 issues the MMAs (kind::f16, M = 128, N = (5 - i) 48)
// into two tensor-memory buffers of five accumulators, and warps 2-9 (two per lane
// quadrant) add the orders in double-float, scale them and store S as
// double-float pairs (the layout the trial kernels read with s_is_df), each warp
// writing 32 consecutive entries of a row of S at a time.  Every mbarrier wait is
// bounded: a block that gives up sets STATUS_TIMEOUT, lets its copies and MMAs
// complete (a fixed bound), frees its tensor memory and returns.
#include <algorithm>

#include "digits.cuh"
#include "kernels.cuh"
#include "tcgen05.cuh"

namespace afq {

namespace {

constexpr int SP_THREADS = 320;            // warp 0 producer, warp 1 MMA issue, warps 2-9 epilogue
constexpr int SP_EPI = 256;
constexpr int SP_NB = 48;                  // proposals per block
constexpr int SP_ORD = 5;                  // accumulators: digit orders 0 .. 4
constexpr int SP_STAGES = 4;
constexpr uint32_t SP_TILE = 16384;        // one digit of U: 128 columns e x 64 K values
constexpr uint32_t SP_BKB = (uint32_t)DG_DIG * SP_NB * 128u;   // one K block of the proposals' digits
constexpr uint32_t SP_DCOLS = (uint32_t)SP_ORD * SP_NB;         // one tensor-memory buffer
constexpr uint32_t SP_TALLOC = 512;

inline size_t sp_smem(int kblk) { return 1024 + (size_t)kblk * SP_BKB + (size_t)SP_STAGES * SP_TILE; }

__device__ __forceinline__ bool sp_wait(uint64_t* bar, uint32_t parity, uint32_t lim, volatile int* fail) {
    if (*fail) return false;
    if (tc::mbar_wait(bar, parity, lim)) return true;
    *fail = 1;
    return false;
}

// fU[e]: exponent of column e of U (its largest |U_k[e]| into [128, 256)).
__global__ void sprop_u_exp_kernel(int K, long long NN, const double* __restrict__ U, int* __restrict__ fU) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < NN; e += (long long)gridDim.x * blockDim.x) {
        float m = 0.f;
        for (int k = 0; k < K; ++k) m = fmaxf(m, fabsf((float)U[(long long)k * NN + e]));
        fU[e] = dg_exp(m);
    }
}

// Uimg[((t KBLK + kb) 5 + i) SP_TILE]: digit i of U columns 128 t .. 128 t + 127,
// K values 64 kb .. 64 kb + 63, K-major in the 128-byte swizzle (zero outside
// K x NN).  One thread per unit (column e, 8 K values).
__global__ void sprop_u_digits_kernel(int K, long long NN, int KBLK, int NTILE, const double* __restrict__ U,
                                      const int* __restrict__ fU, uint8_t* __restrict__ Uimg) {
    const long long units = (long long)NTILE * KBLK * 128 * 8;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < units;
         x += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(x % 128), u = (int)((x / 128) % 8), kb = (int)((x / 1024) % KBLK);
        const long long t = x / (1024LL * KBLK);
        const long long e = t * 128 + r;
        const float sc = e < NN ? dg_p2f(fU[e]) : 0.f;
        uint16_t dg[DG_DIG][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = kb * 64 + 8 * u + q;
            const dfl v = (e < NN && k < K) ? df_from(U[(long long)k * NN + e]) : dfl{0.f, 0.f};
            uint16_t dd[DG_DIG];
            dg_digits(v.hi * sc, v.lo * sc, dd);
#pragma unroll
            for (int i = 0; i < DG_DIG; ++i) dg[i][q] = dd[i];
        }
        uint8_t* base = Uimg + ((size_t)t * KBLK + kb) * DG_DIG * SP_TILE + dg_swz(r, 8 * u);
#pragma unroll
        for (int i = 0; i < DG_DIG; ++i) *reinterpret_cast<uint4*>(base + (size_t)i * SP_TILE) = dg_pack8(dg[i]);
    }
}

}  // namespace

namespace {

__global__ void __launch_bounds__(SP_THREADS, 1)
    sprop_tc_kernel(long long M, int K, long long NN, int KBLK, int NTILE, const double* __restrict__ X,
                    const uint8_t* __restrict__ Uimg, const int* __restrict__ fU, dfl* __restrict__ S, int* status,
                    uint32_t lim) {
    extern __shared__ uint8_t sp_raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)sp_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* BD = sm;                                    // KBLK x SP_BKB: digit j of proposal p at row j 48 + p
    uint8_t* ring = sm + (size_t)KBLK * SP_BKB;          // SP_STAGES x SP_TILE
    __shared__ uint64_t full_bar[SP_STAGES], empty_bar[SP_STAGES], dfull[2], dempty[2], drain_bar;
    __shared__ int erow[SP_NB];
    __shared__ uint32_t tslot;
    __shared__ volatile int fail;

    const long long p0 = (long long)blockIdx.x * SP_NB;
    const int np = (int)min((long long)SP_NB, M - p0);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 1) {
        tc::tmem_alloc(&tslot, SP_TALLOC);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < SP_STAGES; ++q) {
            tc::mbar_init(&full_bar[q], 1);
            tc::mbar_init(&empty_bar[q], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&dfull[b], 1);
            tc::mbar_init(&dempty[b], 1);
        }
        tc::mbar_init(&drain_bar, 1);
        tc::mbar_fence_init();
        fail = 0;
    }
    // row exponents of the block's proposals
    if (tid < SP_NB) {
        float mx = 0.f;
        if (tid < np)
            for (int k = 0; k < K; ++k) mx = fmaxf(mx, fabsf((float)X[(p0 + tid) * K + k]));
        erow[tid] = dg_exp(mx);
    }
    __syncthreads();
    // digits of the proposals: unit (proposal p, K values 8u .. 8u + 7 of block kb)
    for (int x = tid; x < KBLK * SP_NB * 8; x += SP_THREADS) {
        const int p = x % SP_NB, u = (x / SP_NB) % 8, kb = x / (SP_NB * 8);
        const float sc = dg_p2f(erow[p]);
        uint16_t dg[DG_DIG][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = kb * 64 + 8 * u + q;
            const dfl v = (p < np && k < K) ? df_from(X[(p0 + p) * K + k]) : dfl{0.f, 0.f};
            uint16_t dd[DG_DIG];
            dg_digits(v.hi * sc, v.lo * sc, dd);
#pragma unroll
            for (int j = 0; j < DG_DIG; ++j) dg[j][q] = dd[j];
        }
#pragma unroll
        for (int j = 0; j < DG_DIG; ++j)
            *reinterpret_cast<uint4*>(BD + (size_t)kb * SP_BKB + dg_swz(j * SP_NB + p, 8 * u)) = dg_pack8(dg[j]);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    bool failed = false;
    // unit v = (column tile v / (5 KBLK), digit (v / KBLK) % 5, K block v % KBLK)
    const int n_units = NTILE * DG_DIG * KBLK;

    if (warp == 0) {
        // ---- producer
        if (lane == 0) {
            int issued = 0;
            for (int v = 0; v < n_units; ++v) {
                const int st = v % SP_STAGES;
                if (v >= SP_STAGES && !sp_wait(&empty_bar[st], (uint32_t)(((v / SP_STAGES) - 1) & 1), lim, &fail)) {
                    failed = true;
                    break;
                }
                const int t = v / (DG_DIG * KBLK), i = (v / KBLK) % DG_DIG, kb = v % KBLK;
                tc::mbar_arrive_expect_tx(&full_bar[st], SP_TILE);
                tc::bulk_g2s(ring + (size_t)st * SP_TILE, Uimg + (((size_t)t * KBLK + kb) * DG_DIG + i) * SP_TILE,
                             SP_TILE, &full_bar[st]);
                ++issued;
            }
            for (int v = max(0, issued - SP_STAGES); v < issued; ++v)   // every copy lands before the block leaves
                tc::mbar_wait(&full_bar[v % SP_STAGES], (uint32_t)((v / SP_STAGES) & 1), 1u << 22);
            if (failed) atomicOr(status, STATUS_TIMEOUT);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issue (one thread)
        if (lane == 0) {
            int v = 0, committed = 0;
            const uint32_t bbase = tc::smem_u32(BD), rbase = tc::smem_u32(ring);
            for (int t = 0; t < NTILE && !failed; ++t) {
                const int b = t & 1;
                if (t >= 2 && !sp_wait(&dempty[b], (uint32_t)(((t >> 1) - 1) & 1), lim, &fail)) {
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t dbase = taddr + (uint32_t)b * SP_DCOLS;
                for (int i = 0; i < DG_DIG && !failed; ++i) {
                    // digit i of U against the proposals' digits 0 .. 4 - i, into accumulators i .. 4
                    const uint32_t idesc = tc::idesc_f16_f32(128, (SP_ORD - i) * SP_NB);
                    for (int kb = 0; kb < KBLK; ++kb, ++v) {
                        const int st = v % SP_STAGES;
                        if (!sp_wait(&full_bar[st], (uint32_t)((v / SP_STAGES) & 1), lim, &fail)) {
                            failed = true;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t pa = rbase + (uint32_t)st * SP_TILE, pb = bbase + (uint32_t)kb * SP_BKB;
#pragma unroll
                        for (int s = 0; s < 4; ++s) {
                            const uint32_t acc = (i == 0 && kb == 0 && s == 0) ? 0u : 1u;
                            tc::mma_f16(dbase + (uint32_t)(i * SP_NB), tc::desc_sw128(pa + 32u * s),
                                        tc::desc_sw128(pb + 32u * s), idesc, acc);
                        }
                        tc::mma_commit(&empty_bar[st]);
                        ++committed;
                    }
                }
                if (!failed) tc::mma_commit(&dfull[b]);
            }
            if (failed) atomicOr(status, STATUS_TIMEOUT);
            tc::mma_commit(&drain_bar);                  // every issued MMA completes before the block leaves
            tc::mbar_wait(&drain_bar, 0, 1u << 22);
            for (int u = max(0, committed - SP_STAGES); u < committed; ++u)
                tc::mbar_wait(&empty_bar[u % SP_STAGES], (uint32_t)((u / SP_STAGES) & 1), 1u << 22);
        }
        __syncwarp();
    } else {
        // ---- epilogue (warps 2-9): lane r = column e = 128 t + r of the tile; half h of the
        // warps takes the chunks c = h, h + 2, .. of 8 proposals
        const int et = tid - 64;
        const int quad = warp & 3, half = et >> 7;
        const int r = 32 * quad + lane;
        const uint32_t lb = taddr + ((uint32_t)(32 * quad) << 16);
        for (int t = 0; t < NTILE; ++t) {
            const int b = t & 1;
            const bool ok = sp_wait(&dfull[b], (uint32_t)((t >> 1) & 1), lim, &fail);
            if (tc::named_sync_or<SP_EPI>(!ok)) {
                failed = true;
                break;
            }
            tc::fence_after_sync();
            const long long e = (long long)t * 128 + r;
            const float sf = e < NN ? dg_p2f(-fU[e]) : 0.f;
            for (int c = half; c < SP_NB / 8; c += 2) {   // uniform across the warp
                float v[SP_ORD][8];
#pragma unroll
                for (int q = 0; q < SP_ORD; ++q)
                    tc::tmem_ld8(lb + (uint32_t)b * SP_DCOLS + (uint32_t)(q * SP_NB + 8 * c), v[q]);
                tc::tmem_ld_wait();
                if (e < NN) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int p = 8 * c + k;
                        if (p < np) {
                            const dfl z = dg_combine5(v[0][k], v[1][k], v[2][k], v[3][k], v[4][k]);
                            const float f = dg_p2f(-erow[p]);
                            S[(p0 + p) * NN + e] = dfl{z.hi * f * sf, z.lo * f * sf};
                        }
                    }
                }
            }
            // buffer b has been read
            tc::fence_before_sync();
            tc::named_sync<SP_EPI>();
            if (et == 0) tc::mbar_arrive(&dempty[b]);
        }
        if (failed && et == 0) atomicOr(status, STATUS_TIMEOUT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(taddr, SP_TALLOC);
}

}  // namespace

bool sprop_tc_supported(int K, long long NN) { return K >= 1 && K <= 128 && NN >= 1; }

size_t sprop_u_image_bytes(int K, long long NN) {
    const long long ntile = (NN + 127) / 128;
    const int kblk = (K + 63) / 64;
    return (size_t)ntile * kblk * DG_DIG * SP_TILE + (size_t)NN * sizeof(int);
}

cudaError_t sprop_u_images(cudaStream_t s, int K, long long NN, const double* U, void* img) {
    if (!sprop_tc_supported(K, NN)) return cudaErrorInvalidValue;
    const int ntile = (int)((NN + 127) / 128), kblk = (K + 63) / 64;
    uint8_t* Uimg = static_cast<uint8_t*>(img);
    int* fU = reinterpret_cast<int*>(Uimg + (size_t)ntile * kblk * DG_DIG * SP_TILE);
    sprop_u_exp_kernel<<<(unsigned)std::min<long long>((NN + 255) / 256, 4096), 256, 0, s>>>(K, NN, U, fU);
    const long long units = (long long)ntile * kblk * 1024;
    sprop_u_digits_kernel<<<(unsigned)std::min<long long>((units + 255) / 256, 8192), 256, 0, s>>>(K, NN, kblk, ntile,
                                                                                                    U, fU, Uimg);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t sprop_tc(cudaStream_t s, long long M, int K, long long NN, const double* X, const void* img, void* S,
                     int* status, uint32_t lim) {
    if (M <= 0) return cudaSuccess;
    if (!sprop_tc_supported(K, NN)) return cudaErrorInvalidValue;
    const int ntile = (int)((NN + 127) / 128), kblk = (K + 63) / 64;
    const uint8_t* Uimg = static_cast<const uint8_t*>(img);
    const int* fU = reinterpret_cast<const int*>(Uimg + (size_t)ntile * kblk * DG_DIG * SP_TILE);
    const size_t smem = sp_smem(kblk);
    cudaError_t e = raise_smem_limit((const void*)sprop_tc_kernel, smem);
    if (e != cudaSuccess) return e;
    sprop_tc_kernel<<<(unsigned)((M + SP_NB - 1) / SP_NB), SP_THREADS, smem, s>>>(
        M, K, NN, kblk, ntile, X, Uimg, fU, static_cast<dfl*>(S), status, lim ? lim : (1u << 26));
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace afq
