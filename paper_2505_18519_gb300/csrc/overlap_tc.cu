// Overlap matrices A_p = Phi_p^T phi_w of every pair of a walker (<Phi_p|phi> =
// det A_p per spin for a real trial: the path signs of Eq. (26) and the ratios of
// Eq. (25)) on the tensor cores, for the mixed-precision path; the LU,
// log-determinant and inverse stay in overlap_lu.
//
// For one walker and spin (n electrons) the products of all P paths are one GEMM
//   D[(p, a), (b, ri)] = sum_i Phi_p[i, a] Re/Im phi_w[i, b],
// 128-row tiles of PB = 128 / n pairs, K = i in blocks of 64.  Both operands are
// split error-free into five 8-bit digits (digits.cuh) from their double-float
// copies, A rows (p, a) scaled by 2^erow so that each row's largest entry lies in
// [128, 256), B rows (b, ri) by 2^fcol the same way.  One MMA of digit i of A
// against the digits 0 .. 4 - i of B laid side by side (rows j CB + c) adds
// A_i B_j to accumulator i + j for every j at once; the orders 0 .. 4 (15 digit
// products) are kept.  For N <= 128 every partial sum of an accumulator is an
// integer of magnitude at most (2 * 256 * 129 + 3 * 129^2) * 128 < 1.5e7 < 2^24
// (order 4, the largest), so the tensor cores add exactly; larger N is left to
// the double-float kernel.  The dropped orders and the digits' truncation bound
// an entry's error by about 2^-38 of max_i |Phi_ia| max_i |phi_ib| N: about 40
// bits, against about 44 for the compensated double-float sums.
//
// Block: walker blockIdx.x / MT, tile blockIdx.x % MT of its pairs; 256 threads.
// Per K block all threads write the digits of both operands into shared memory,
// thread 0 issues the MMAs (kind::f16, M = 128, accumulators in tensor memory:
// order q at columns q CB .. q CB + CB - 1, CB = 2n rounded up to 16), and the
// block waits for them before the next K block overwrites the digits.  The
// epilogue (eight warps, two per tensor-memory lane quadrant) adds the orders in
// double-float and writes A as (Re hi, Re lo, Im hi, Im lo) per entry.
// Every mbarrier wait is bounded: a block that gives up sets STATUS_TIMEOUT,
// waits (a fixed bound) for its own MMAs, frees its tensor memory and returns.
#include <algorithm>

#include "digits.cuh"
#include "kernels.cuh"
#include "tcgen05.cuh"

namespace afq {

namespace {

constexpr int OT_THREADS = 256;
constexpr int OT_ORD = 5;                  // accumulators: digit orders 0 .. 4
constexpr uint32_t OT_AKB = 16384;         // one digit of A for one K block: 128 rows x 128 bytes

__host__ __device__ inline int ot_cb(int n) { return (2 * n + 15) / 16 * 16; }
// one K block of the B digits: DG_DIG blocks of CB rows of 128 bytes
__host__ __device__ inline uint32_t ot_bkb(int cb) { return (uint32_t)DG_DIG * (uint32_t)cb * 128u; }
inline size_t ot_smem(int cb) { return 1024 + (size_t)DG_DIG * OT_AKB + ot_bkb(cb); }
inline uint32_t ot_talloc(int cb) {
    const int cols = OT_ORD * cb;
    return cols <= 32 ? 32u : (cols <= 64 ? 64u : (cols <= 128 ? 128u : (cols <= 256 ? 256u : 512u)));
}

}  // namespace

__global__ void __launch_bounds__(OT_THREADS)
    overlap_tc_kernel(int N, int nu, int nt, int n, int col0, int P, int PB, int MT, int KBLK, int CB,
                      const dfl* __restrict__ PhiD, long long Phi_stride, const float4* __restrict__ phiD,
                      const int* __restrict__ alive, float4* __restrict__ Aout, int* status, uint32_t talloc,
                      uint32_t lim) {
    extern __shared__ uint8_t ot_raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)ot_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* AD = sm;                                  // digit q of rows (p_l, a): AD + q OT_AKB
    uint8_t* BD = sm + (size_t)DG_DIG * OT_AKB;        // digit j of row c = (b, ri): row j CB + c
    __shared__ int erow[128], fcol[128];
    __shared__ uint64_t mma_bar;
    __shared__ uint32_t tslot;

    const long long w = blockIdx.x / MT;
    const int m = blockIdx.x % MT;
    if (alive && !alive[w]) return;                    // uniform: before any allocation
    const int np = min(PB, P - m * PB);
    const int rows = np * n;
    const long long pair0 = w * P + (long long)m * PB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float4* ph = phiD + w * (long long)N * nt + col0;   // phi_w[i, b] at ph[i nt + b]

    if (warp == 0) {
        tc::tmem_alloc(&tslot, talloc);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&mma_bar, 1);
        tc::mbar_fence_init();
    }
    // row and column exponents: the largest |entry| of each operand row into [128, 256)
    if (tid < 128) {
        float mx = 0.f;
        if (tid < rows) {
            const int pl = tid / n, a = tid - pl * n;
            const dfl* Pp = PhiD + (pair0 + pl) * Phi_stride + a;
            for (int i = 0; i < N; ++i) mx = fmaxf(mx, fabsf(Pp[(long long)i * nu].hi));
        }
        erow[tid] = dg_exp(mx);
    } else if (tid - 128 < CB) {
        const int c = tid - 128;
        float mx = 0.f;
        if (c < 2 * n) {
            for (int i = 0; i < N; ++i) {
                const float4 g = ph[(long long)i * nt + (c >> 1)];
                mx = fmaxf(mx, fabsf((c & 1) ? g.z : g.x));
            }
        }
        fcol[c] = dg_exp(mx);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    const int maxblk = 256 / CB;                       // B digit blocks per MMA (N <= 256)
    bool failed = false;
    int issued = 0;                                    // K blocks whose products were issued
    for (int kb = 0; kb < KBLK; ++kb) {
        if (kb > 0) {   // the products of the previous K block have read the digits
            const bool ok = tc::mbar_wait(&mma_bar, (uint32_t)((kb - 1) & 1), lim);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            tc::fence_after_sync();
        }
        // digits of A: unit (row r, K values 8u .. 8u + 7 of this block)
        for (int e = tid; e < 128 * 8; e += OT_THREADS) {
            const int r = e & 127, u = e >> 7;
            const float sc = dg_p2f(erow[r]);
            const dfl* Pp = nullptr;
            if (r < rows) {
                const int pl = r / n, a = r - pl * n;
                Pp = PhiD + (pair0 + pl) * Phi_stride + a;
            }
            uint16_t dg[DG_DIG][8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int i = kb * 64 + 8 * u + t;
                const dfl x = (Pp && i < N) ? Pp[(long long)i * nu] : dfl{0.f, 0.f};
                uint16_t dd[DG_DIG];
                dg_digits(x.hi * sc, x.lo * sc, dd);
#pragma unroll
                for (int q = 0; q < DG_DIG; ++q) dg[q][t] = dd[q];
            }
            const uint32_t off = dg_swz(r, 8 * u);
#pragma unroll
            for (int q = 0; q < DG_DIG; ++q) *reinterpret_cast<uint4*>(AD + (size_t)q * OT_AKB + off) = dg_pack8(dg[q]);
        }
        // digits of B: unit (column c = (b, ri), K values 8u .. 8u + 7); rows c >= 2n zero
        for (int e = tid; e < CB * 8; e += OT_THREADS) {
            const int c = e % CB, u = e / CB;
            const float sc = dg_p2f(fcol[c]);
            uint16_t dg[DG_DIG][8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int i = kb * 64 + 8 * u + t;
                float h = 0.f, l = 0.f;
                if (c < 2 * n && i < N) {
                    const float4 g = ph[(long long)i * nt + (c >> 1)];
                    h = (c & 1) ? g.z : g.x;
                    l = (c & 1) ? g.w : g.y;
                }
                uint16_t dd[DG_DIG];
                dg_digits(h * sc, l * sc, dd);
#pragma unroll
                for (int q = 0; q < DG_DIG; ++q) dg[q][t] = dd[q];
            }
#pragma unroll
            for (int j = 0; j < DG_DIG; ++j)
                *reinterpret_cast<uint4*>(BD + dg_swz(j * CB + c, 8 * u)) = dg_pack8(dg[j]);
        }
        tc::fence_proxy_async();   // the digits, written by the threads, to the tensor cores
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            const uint32_t abase = tc::smem_u32(AD), bbase = tc::smem_u32(BD);
            for (int s = 0; s < 4; ++s) {
#pragma unroll
                for (int i = 0; i < DG_DIG; ++i) {
                    // digit i of A against B digits 0 .. 4 - i, into accumulators i .. 4 (digit
                    // 0 first: at the block's first K step it initialises every accumulator)
                    const int nblk = OT_ORD - i;
                    const uint64_t ad = tc::desc_sw128(abase + (uint32_t)i * OT_AKB + 32u * s);
                    for (int j0 = 0; j0 < nblk; j0 += maxblk) {
                        const int nb = min(maxblk, nblk - j0);
                        const uint64_t bd = tc::desc_sw128(bbase + (uint32_t)(j0 * CB) * 128u + 32u * s);
                        const uint32_t acc = (kb == 0 && s == 0 && i == 0) ? 0u : 1u;
                        tc::mma_f16(taddr + (uint32_t)((i + j0) * CB), ad, bd, tc::idesc_f16_f32(128, nb * CB), acc);
                    }
                }
            }
            tc::mma_commit(&mma_bar);
        }
        ++issued;
    }
    if (!failed) {
        const bool ok = tc::mbar_wait(&mma_bar, (uint32_t)((KBLK - 1) & 1), lim);
        if (__syncthreads_or(!ok)) failed = true;
        tc::fence_after_sync();
    }
    if (!failed) {
        // epilogue: lane r = (p_l, a) of a quadrant; half h of the warps takes the column
        // chunks t = h, h + 2, .. of 8 columns (four entries b, Re and Im side by side)
        const int quad = warp & 3, half = warp >> 2;
        const int r = 32 * quad + lane;
        const bool row_ok = r < rows;
        const int pl = row_ok ? r / n : 0, a = row_ok ? r - pl * n : 0;
        const float srow = dg_p2f(-erow[r]);
        float4* Ap = Aout + ((pair0 + pl) * n + a) * (long long)n;
        const uint32_t lb = taddr + ((uint32_t)(32 * quad) << 16);
        const int nch = (2 * n + 7) / 8;
        for (int t = half; t < nch; t += 2) {       // uniform across the warp
            float v[OT_ORD][8];
#pragma unroll
            for (int q = 0; q < OT_ORD; ++q) tc::tmem_ld8(lb + (uint32_t)(q * CB + 8 * t), v[q]);
            tc::tmem_ld_wait();
            if (row_ok) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int b = 4 * t + k;
                    if (b < n) {
                        const dfl re = dg_combine5(v[0][2 * k], v[1][2 * k], v[2][2 * k], v[3][2 * k], v[4][2 * k]);
                        const dfl im = dg_combine5(v[0][2 * k + 1], v[1][2 * k + 1], v[2][2 * k + 1], v[3][2 * k + 1],
                                                   v[4][2 * k + 1]);
                        const float sr = dg_p2f(-fcol[2 * b]), si = dg_p2f(-fcol[2 * b + 1]);
                        Ap[b] = make_float4(re.hi * srow * sr, re.lo * srow * sr, im.hi * srow * si, im.lo * srow * si);
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(status, STATUS_TIMEOUT);
        if (issued > 0) tc::mbar_wait(&mma_bar, (uint32_t)((issued - 1) & 1), 1u << 22);   // its MMAs complete
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, talloc);
}

bool overlap_tc_supported(int N, int n) { return n >= 1 && n <= 40 && N >= 1 && N <= 128; }

cudaError_t overlap_tc(cudaStream_t s, const Dims& d, const void* PhiD, long long Phi_stride, const void* phiD,
                       const int* alive, void* Aout, int* status) {
    if (d.pairs <= 0) return cudaSuccess;
    float4* out = static_cast<float4*>(Aout);
    const long long W = d.pairs / d.P;
    for (int spin = 0; spin < 2; ++spin) {
        const int n = spin ? d.nd : d.nu;
        if (n == 0) continue;
        if (!overlap_tc_supported(d.N, n) || d.cphi || !PhiD || !phiD) return cudaErrorInvalidValue;
        const int CB = ot_cb(n), PB = std::min(128 / n, d.P), MT = (d.P + PB - 1) / PB;
        const int KBLK = (d.N + 63) / 64;
        const size_t smem = ot_smem(CB);
        cudaError_t e = raise_smem_limit((const void*)overlap_tc_kernel, smem);
        if (e != cudaSuccess) return e;
        overlap_tc_kernel<<<(unsigned)(W * MT), OT_THREADS, smem, s>>>(
            d.N, d.nu, d.nt, n, spin ? d.nu : 0, d.P, PB, MT, KBLK, CB, static_cast<const dfl*>(PhiD), Phi_stride,
            static_cast<const float4*>(phiD), alive, out + (spin ? d.pairs * (long long)d.nu * d.nu : 0), status,
            ot_talloc(CB), d.wait_polls ? d.wait_polls : (1u << 26));
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace afq
